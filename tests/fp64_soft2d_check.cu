// Host-only harness for tests/test_fp64_soft.py: the integer-pipe FP64 update of the 2D heat
// kernels (soft64::heat2d_update in csrc/fp64_soft2d.cuh, compiled here as host code) against the
// host's own IEEE 754 binary64 arithmetic,
//   fma(rx, fma(-2, u, a + b), fma(ry, fma(-2, u, d + e), u))
// with std::fma and no contraction. Every case the integer path accepts must give the same bits.
//
// usage: fp64_soft2d_check seed cases_per_family
// prints one line per family: name cases fast mismatches; exit 1 on any mismatch.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "fp64_soft2d.cuh"

using namespace sw;

static std::mt19937_64 rng;
static long g_bad = 0;

struct Count {
    long cases = 0, fast = 0, bad = 0;
};

static double ieee(double rx, double ry, double a, double b, double u, double d, double e) {
    return std::fma(rx, std::fma(-2.0, u, a + b), std::fma(ry, std::fma(-2.0, u, d + e), u));
}

static void check(Count &c, double rx, double ry, double a, double b, double u, double d, double e) {
    const soft64::HeatR hx = soft64::make_heat_r(rx), hy = soft64::make_heat_r(ry);
    bool ok = true;
    const uint64_t got = soft64::heat2d_update(hx, hy, soft64::bits(a), soft64::bits(b), soft64::bits(u),
                                               soft64::bits(d), soft64::bits(e), ok);
    ++c.cases;
    if (!ok) return;
    ++c.fast;
    const double want = ieee(rx, ry, a, b, u, d, e);
    if (got != soft64::bits(want)) {
        if (g_bad++ < 8)
            std::printf("mismatch rx=%a ry=%a a=%a b=%a u=%a d=%a e=%a: %a, IEEE %a\n", rx, ry, a, b, u, d, e,
                        soft64::value(got), want);
        ++c.bad;
    }
}

// random sign and significand, biased exponent in [lo, hi]
static double rexp(int lo, int hi) {
    std::uniform_int_distribution<int> e(lo, hi);
    return soft64::value((rng() & soft64::kFrac) | ((uint64_t)e(rng) << 52) | (rng() & soft64::kSign));
}
// u (1 + t 2^-scale), t uniform in [-1, 1)
static double near(double u, int scale) {
    return u * (1.0 + std::ldexp((double)((int64_t)(rng() >> 11) - (1LL << 52)), -52 - scale));
}

static void report(const char *name, const Count &c) {
    std::printf("%s %ld %ld %ld\n", name, c.cases, c.fast, c.bad);
}

int main(int argc, char **argv) {
    rng.seed(argc > 1 ? std::strtoull(argv[1], nullptr, 10) : 1);
    const long N = argc > 2 ? std::atol(argv[2]) : 1000000;
    std::uniform_real_distribution<double> ur(0.01, 0.25);
    {   // all four neighbours close to u, each direction at its own relative scale
        Count c;
        for (long i = 0; i < N; ++i) {
            const double u = rexp(1000, 1040);
            const int sx = (int)(rng() % 50), sy = (int)(rng() % 50);
            check(c, ur(rng), ur(rng), near(u, sx), near(u, sx), u, near(u, sy), near(u, sy));
        }
        report("smooth", c);
    }
    {   // one neighbour per direction 2^0 .. 2^-9 of u (across the low edge of the exponent
        // window), its partner about 2u minus it, so that the second difference stays small
        Count c;
        for (long i = 0; i < N; ++i) {
            const double u = rexp(1020, 1026);
            double n4[4];
            for (int k = 0; k < 2; ++k) {
                const double p = near(std::ldexp(u, -(int)(rng() % 10)), 2);
                const double q = near(2.0 * u - p, 20 + (int)(rng() % 30));
                n4[2 * k] = (rng() & 1) ? p : q;
                n4[2 * k + 1] = n4[2 * k] == p ? q : p;
            }
            check(c, ur(rng), ur(rng), n4[0], n4[1], u, n4[2], n4[3]);
        }
        report("window", c);
    }
    {   // exact ties: in the inner rounding (ry = 2^-j, ry yd = (K + 1/2) ulp(u), x flat), in the
        // outer one (rx = 2^-j, y flat), and in the outer one after an exact inner correction of
        // either parity (the tie then goes to the even neighbour of the inner result, not of u)
        Count c;
        for (long i = 0; i < N; ++i) {
            const int j = 1 + (int)(rng() % 6);
            const double u = std::fabs(rexp(1023, 1023)) * ((rng() & 1) ? 1 : -1);
            const double ulp = std::ldexp(1.0, std::ilogb(u) - 52);
            const uint64_t K = rng() >> 34;
            double dd = std::ldexp((double)(2 * K + 1), j - 1) * ulp;
            if (rng() & 1) dd = -dd;
            const double r = std::ldexp(1.0, -j);
            switch (rng() % 3) {
            case 0: check(c, ur(rng), r, u, u, u, u + dd, u); break;
            case 1: check(c, r, ur(rng), u + dd, u, u, u, u); break;
            default: {
                const int j2 = 1 + (int)(rng() % 6);
                const uint64_t K2 = 1 + (rng() >> 40);
                double dy = std::ldexp((double)K2, j2) * ulp;  // ry yd = K2 ulp(u) exactly
                if (rng() & 1) dy = -dy;
                check(c, r, std::ldexp(1.0, -j2), u + dd, u, u, u + dy, u);
            }
            }
        }
        report("ties", c);
    }
    {   // u at the edges of its binade, so that either correction may leave it
        Count c;
        for (long i = 0; i < N; ++i) {
            const uint64_t frac = (rng() & 1) ? rng() % 1024 : soft64::kFrac - rng() % 1024;
            const double u = soft64::value(((uint64_t)(1021 + rng() % 5) << 52) | frac | (rng() & soft64::kSign));
            const int sx = 20 + (int)(rng() % 30), sy = 20 + (int)(rng() % 30);
            check(c, ur(rng), ur(rng), near(u, sx), near(u, sx), u, near(u, sy), near(u, sy));
        }
        report("binade", c);
    }
    {   // multipliers with few significant bits (the products' low bits vanish), across their range
        Count c;
        for (long i = 0; i < N; ++i) {
            const double rx = std::ldexp((double)(1 + rng() % 16), -(int)(rng() % 30) - 4);
            const double ry = std::ldexp((double)(1 + rng() % 16), -(int)(rng() % 30) - 4);
            const double u = rexp(1010, 1030);
            const int sx = (int)(rng() % 40), sy = (int)(rng() % 40);
            check(c, rx, ry, near(u, sx), near(u, sx), u, near(u, sy), near(u, sy));
        }
        report("r_bits", c);
    }
    {   // anything: zeros, subnormals, infinities, NaNs, extreme exponents, mixed signs
        Count c;
        for (long i = 0; i < N; ++i)
            check(c, ur(rng), ur(rng), soft64::value(rng()), soft64::value(rng()), soft64::value(rng()),
                  soft64::value(rng()), soft64::value(rng()));
        for (long i = 0; i < N; ++i) {
            const double u = rexp(1, 80);
            check(c, ur(rng), ur(rng), near(u, 3), near(u, 3), u, near(u, 3), near(u, 3));
        }
        for (long i = 0; i < N; ++i) {
            const double u = rexp(2030, 2046);
            check(c, ur(rng), ur(rng), near(u, 3), near(u, 3), u, near(u, 3), near(u, 3));
        }
        for (long i = 0; i < N; ++i) {
            const double u = rexp(1023, 1023);
            check(c, ur(rng), ur(rng), 0.0, u, u, (rng() & 1) ? -u : u, u);
        }
        report("special", c);
    }
    {   // the 2D heat run itself: a periodic 96 x 64 field of separable modes, 300 steps
        Count c;
        const int nx = 96, ny = 64;
        const double rx = 0.2137, ry = 0.1713;
        const soft64::HeatR hx = soft64::make_heat_r(rx), hy = soft64::make_heat_r(ry);
        std::vector<double> x(nx * ny), y(nx * ny);
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double t = 1.5;
                for (int m = 1; m <= 6; ++m)
                    t += std::sin(2 * M_PI * (m * 5 % 11) * i / nx + m) * std::cos(2 * M_PI * (m * 3 % 7) * j / ny) *
                         (((m * 13) % 7) - 3) / 9.0;
                x[j * nx + i] = t;
            }
        for (int step = 0; step < 300; ++step) {
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    const double a = x[j * nx + (i + nx - 1) % nx], b = x[j * nx + (i + 1) % nx], u = x[j * nx + i];
                    const double d = x[((j + ny - 1) % ny) * nx + i], e = x[((j + 1) % ny) * nx + i];
                    const double want = ieee(rx, ry, a, b, u, d, e);
                    bool ok = true;
                    const uint64_t got = soft64::heat2d_update(hx, hy, soft64::bits(a), soft64::bits(b),
                                                               soft64::bits(u), soft64::bits(d), soft64::bits(e), ok);
                    ++c.cases;
                    if (ok) {
                        ++c.fast;
                        if (got != soft64::bits(want)) ++c.bad, ++g_bad;
                    }
                    y[j * nx + i] = want;
                }
            std::swap(x, y);
        }
        report("heat_run", c);
    }
    return g_bad ? 1 : 0;
}
