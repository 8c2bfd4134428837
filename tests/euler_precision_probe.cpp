// euler_precision_probe.cpp -- test infrastructure: where the FP32 error of the Euler scheme
// comes from. The scheme of the oracle's reading (pressure-ratio minmod limiter, Rusanov
// flux, two-stage step; Sections 4.2-4.3) restated once more, templated on the arithmetic,
// and run in variants that move single steps between FP32 and FP64. Shares no code with
// the library or the oracle; compiled by tests/test_euler_precision_probe.py with
// -ffp-contract=off. Output: one line per variant, "name rho_max rho_l2 min_rho min_p".
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <algorithm>

template <class T> struct K { T gamma, gm1, lam, hlam; };

template <class T> T pres(const K<T>& k, T r, T m, T E) { T u = m / r; return k.gm1 * (E - (T(0.5) * m) * u); }
template <class T> T ratio(T pm, T p0, T pp) {
  T dm = p0 - pm, dp = pp - p0;
  if ((dm > 0 && dp > 0) || (dm < 0 && dp < 0)) return dm / dp;
  return 0;
}
template <class T> void phys(const K<T>& k, T r, T m, T E, T& f0, T& f1, T& f2, T& s) {
  T u = m / r; T p = k.gm1 * (E - (T(0.5) * m) * u); T c = std::sqrt((k.gamma * p) / r);
  f0 = m; f1 = m * u + p; f2 = (E + p) * u; s = std::fabs(u) + c;
}
template <class T> void face(const K<T>& k, const T* a, T tha, const T* b, T thb, T* o) {
  T phl = tha < 1 ? tha : T(1);
  T phr = thb > 1 ? T(1) / thb : (thb > 0 ? T(1) : T(0));
  T hl = T(0.5) * phl, hr = T(0.5) * phr;
  T l[3], rr[3];
  for (int v = 0; v < 3; ++v) { T d = b[v] - a[v]; l[v] = a[v] + hl * d; rr[v] = b[v] - hr * d; }
  T fl[3], fr[3], sl, sr;
  phys(k, l[0], l[1], l[2], fl[0], fl[1], fl[2], sl);
  phys(k, rr[0], rr[1], rr[2], fr[0], fr[1], fr[2], sr);
  T s = sl > sr ? sl : sr, hs = T(0.5) * s;
  for (int v = 0; v < 3; ++v) o[v] = T(0.5) * (fl[v] + fr[v]) - hs * (rr[v] - l[v]);
}
static void two_sum(float a, float b, float& s, float& e) { s = a + b; float bb = s - a; float aa = s - bb; e = (a - aa) + (b - bb); }
static void fast2(float a, float b, float& s, float& e) { s = a + b; e = b - (s - a); }

// mode: 0 FP64; 1 FP32; 2 FP32 hi/lo state, pressure, ratio and flux from the high parts
// (the library's FP32_COMP); 3 as 2 with pressure and ratio in FP64 from hi + lo (Q* kept as
// a hi/lo pair); 4 FP32 with pressure and ratio in FP64; 6 hi/lo state with every step in
// FP64; 7 hi/lo state with the flux in FP64 but pressure and ratio from the high parts
struct Res { std::vector<double> q[3]; };

Res run(int mode, const std::vector<double>* q0, int n, double lam, int steps, bool periodic) {
  const double gamma = 1.4;
  K<double> kd{gamma, gamma - 1, lam, 0.5 * lam};
  K<float> kf{(float)gamma, (float)(gamma - 1), (float)lam, (float)(0.5 * lam)};
  Res out;
  auto idx = [&](int i) { if (periodic) return (i + n) % n; return i < 0 ? 0 : (i >= n ? n - 1 : i); };
  auto edge = [&](int i) { return !periodic && (i < 0 || i >= n); };
  if (mode == 0) {
    std::vector<double> Q[3], Qs[3], th(n), p(n), F[3];
    for (int v = 0; v < 3; ++v) { Q[v] = q0[v]; Qs[v].resize(n); F[v].resize(n + 1); }
    for (int s = 0; s < steps; ++s) for (int st = 0; st < 2; ++st) {
      std::vector<double>* src = st == 0 ? Q : Qs;
#pragma omp parallel for
      for (int i = 0; i < n; ++i) p[i] = pres(kd, src[0][i], src[1][i], src[2][i]);
#pragma omp parallel for
      for (int i = 0; i < n; ++i) th[i] = ratio(p[idx(i - 1)], p[i], p[idx(i + 1)]);
#pragma omp parallel for
      for (int f = 0; f <= n; ++f) {  // face between f-1 and f
        int a = idx(f - 1), b = idx(f);
        double qa[3] = {src[0][a], src[1][a], src[2][a]}, qb[3] = {src[0][b], src[1][b], src[2][b]}, o[3];
        double ta = edge(f - 1) ? 0 : th[a], tb = edge(f) ? 0 : th[b];
        face(kd, qa, ta, qb, tb, o);
        for (int v = 0; v < 3; ++v) F[v][f] = o[v];
      }
#pragma omp parallel for
      for (int i = 0; i < n; ++i) for (int v = 0; v < 3; ++v) {
        double d = F[v][i + 1] - F[v][i];
        if (st == 0) Qs[v][i] = Q[v][i] - kd.hlam * d; else Q[v][i] = Q[v][i] - kd.lam * d;
      }
    }
    for (int v = 0; v < 3; ++v) out.q[v] = Q[v];
    return out;
  }
  // float-family modes
  std::vector<float> Qh[3], Ql[3], Sh[3], Sl[3], th(n), F[3];
  std::vector<double> p(n);
  for (int v = 0; v < 3; ++v) {
    Qh[v].resize(n); Ql[v].resize(n); Sh[v].resize(n); Sl[v].resize(n); F[v].resize(n + 1);
    for (int i = 0; i < n; ++i) {
      float h = (float)q0[v][i];
      Qh[v][i] = h; Ql[v][i] = (mode == 2 || mode == 3) ? (float)(q0[v][i] - (double)h) : 0.f;
    }
  }
  const bool comp = mode == 2 || mode == 3 || mode >= 6, p64 = mode == 3 || mode == 4 || mode == 6;
  const bool f64 = mode >= 6;
  std::vector<double> Fd[3];
  for (int v = 0; v < 3; ++v) Fd[v].resize(n + 1);
  for (int s = 0; s < steps; ++s) for (int st = 0; st < 2; ++st) {
    std::vector<float>* H = st == 0 ? Qh : Sh;
    std::vector<float>* L = st == 0 ? Ql : Sl;
    const bool haslo = comp && (st == 0 || mode == 3 || mode >= 6);
#pragma omp parallel for
    for (int i = 0; i < n; ++i) {
      if (p64) {
        double r = (double)H[0][i] + (haslo ? (double)L[0][i] : 0.0);
        double m = (double)H[1][i] + (haslo ? (double)L[1][i] : 0.0);
        double E = (double)H[2][i] + (haslo ? (double)L[2][i] : 0.0);
        p[i] = pres(kd, r, m, E);
      } else p[i] = (double)pres(kf, H[0][i], H[1][i], H[2][i]);
    }
#pragma omp parallel for
    for (int i = 0; i < n; ++i) {
      if (p64) th[i] = (float)ratio(p[idx(i - 1)], p[i], p[idx(i + 1)]);
      else th[i] = ratio((float)p[idx(i - 1)], (float)p[i], (float)p[idx(i + 1)]);
    }
#pragma omp parallel for
    for (int f = 0; f <= n; ++f) {
      int a = idx(f - 1), b = idx(f);
      float ta = edge(f - 1) ? 0.f : th[a], tb = edge(f) ? 0.f : th[b];
      if (f64) {
        double qa[3], qb[3], o[3];
        for (int v = 0; v < 3; ++v) { qa[v] = (double)H[v][a] + (double)L[v][a]; qb[v] = (double)H[v][b] + (double)L[v][b]; }
        face(kd, qa, (double)ta, qb, (double)tb, o);
        for (int v = 0; v < 3; ++v) Fd[v][f] = o[v];
      } else {
        float qa[3] = {H[0][a], H[1][a], H[2][a]}, qb[3] = {H[0][b], H[1][b], H[2][b]}, o[3];
        face(kf, qa, ta, qb, tb, o);
        for (int v = 0; v < 3; ++v) F[v][f] = o[v];
      }
    }
#pragma omp parallel for
    for (int i = 0; i < n; ++i) for (int v = 0; v < 3; ++v) {
      if (f64) {
        double c = st == 0 ? kd.hlam : kd.lam;
        double x = ((double)Qh[v][i] + (double)Ql[v][i]) - c * (Fd[v][i + 1] - Fd[v][i]);
        float h = (float)x, l = (float)(x - (double)h);
        if (st == 0) { Sh[v][i] = h; Sl[v][i] = l; } else { Qh[v][i] = h; Ql[v][i] = l; }
        continue;
      }
      float d = F[v][i + 1] - F[v][i];
      if (!comp) {
        if (st == 0) Sh[v][i] = Qh[v][i] - kf.hlam * d; else Qh[v][i] = Qh[v][i] - kf.lam * d;
      } else if (st == 0 && mode == 2) {
        Sh[v][i] = Qh[v][i] + (Ql[v][i] - kf.hlam * d);
      } else {
        float c = st == 0 ? kf.hlam : kf.lam;
        float delta = -(c * d), sm, e, nh, nl;
        two_sum(Qh[v][i], delta, sm, e);
        fast2(sm, Ql[v][i] + e, nh, nl);
        if (st == 0) { Sh[v][i] = nh; Sl[v][i] = nl; } else { Qh[v][i] = nh; Ql[v][i] = nl; }
      }
    }
  }
  for (int v = 0; v < 3; ++v) { out.q[v].resize(n); for (int i = 0; i < n; ++i) out.q[v][i] = (double)Qh[v][i] + (double)Ql[v][i]; }
  return out;
}

int main(int argc, char** argv) {
  const int n = atoi(argv[1]), steps = atoi(argv[2]), kind = atoi(argv[3]);
  std::vector<double> q0[3];
  for (int v = 0; v < 3; ++v) q0[v].resize(n);
  double lam;
  bool periodic = false;
  if (kind == 0) {  // Sod
    lam = 0.4 / 2.2;
    for (int i = 0; i < n; ++i) { bool L = i < n / 2; double r = L ? 1 : 0.125, p = L ? 1 : 0.1; q0[0][i] = r; q0[1][i] = 0; q0[2][i] = p / 0.4; }
  } else {  // periodic random Riemann segments (a fixed LCG: no library generator)
    lam = 0.4 / 5.0; periodic = true;
    const int nseg = 16;
    unsigned long long s = 12345;
    auto next = [&]() { s = s * 6364136223846793005ULL + 1442695040888963407ULL; return (double)(s >> 11) * 0x1.0p-53; };
    for (int g = 0; g < nseg; ++g) {
      double r = pow(10, -next()), p = pow(10, -next()), u = next() - 0.5;
      for (int i = g * n / nseg; i < (g + 1) * n / nseg; ++i) { q0[0][i] = r; q0[1][i] = r * u; q0[2][i] = p / 0.4 + 0.5 * r * u * u; }
    }
  }
  Res ref = run(0, q0, n, lam, steps, periodic);
  const int modes[] = {1, 2, 3, 4, 5, 6, 7};
  const char* names[] = {"", "fp32", "hilo", "hilo_p64", "fp32_p64", "fp64_1ulp", "hilo_all64", "hilo_flux64"};
  for (int mode : modes) {
    std::vector<double> qp[3];
    for (int v = 0; v < 3; ++v) qp[v] = q0[v];
    if (mode == 5) for (int i = 0; i < n; i += 7) qp[2][i] = nextafter(qp[2][i], 10.0);  // 1 ulp in E
    Res g = run(mode == 5 ? 0 : mode, mode == 5 ? qp : q0, n, lam, steps, periodic);
    double mx = 0, m0 = 0, s2 = 0, o2 = 0, minr = 1e300, minp = 1e300;
    for (int i = 0; i < n; ++i) {
      double d = fabs(g.q[0][i] - ref.q[0][i]);
      mx = std::max(mx, d); m0 = std::max(m0, fabs(ref.q[0][i])); s2 += d * d; o2 += ref.q[0][i] * ref.q[0][i];
      minr = std::min(minr, g.q[0][i]);
      minp = std::min(minp, 0.4 * (g.q[2][i] - 0.5 * g.q[1][i] * g.q[1][i] / g.q[0][i]));
    }
    printf("%s %.6e %.6e %.9g %.9g\n", names[mode], mx / m0, sqrt(s2 / o2), minr, minp);
  }
  return 0;
}
