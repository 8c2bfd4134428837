// Host-only harness for tests/test_host_engine.py: runs every structure of every
// phase of a swept run through the host engine of the hybrid CPU/GPU split
// (csrc/cpu_phase.h) -- as if the host took all tiles -- and writes the final
// state. The test compares it with the oracle. No device code runs.
//
// usage: host_engine_check scheme(0 heat, 1 euler) prec(0 fp64, 1 fp32, 2 hi/lo)
//        n W periodic steps r_or_lambda gamma infile outfile
//   infile / outfile: FP64 planes (heat 1, Euler 3), n doubles each.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "cpu_phase.h"

using namespace sw;

template <class Sch>
static void run(const Sch &sch0, std::vector<typename Sch::T> &st, int64_t n, int W, int periodic, int64_t L) {
    using T = typename Sch::T;
    const int H = W / 2;
    const int64_t M = n / W, S = M + 1;
    const int64_t P_last = (L + H - 1) / H;
    std::vector<T> fl[2];
    fl[0].assign((size_t)Sch::NF * S * 2 * W, T(0));
    fl[1] = fl[0];
    Sch sch = sch0;
    std::vector<T> work(2 * Sch::NF * (W + 2));
    WrittenRange wr;
    for (int64_t p = 0; p <= P_last; ++p) {
        HostPhase<T> a{};
        a.n = n;
        a.W = W;
        a.H = H;
        a.periodic = periodic;
        a.p = (p == 0) ? 0 : (int)(2 - (p & 1));
        a.F = p * H;
        a.lower = (p == 0) ? 0 : (int)std::min<int64_t>(H, L - (p - 1) * H);
        a.upper = (p == P_last) ? 0 : (int)std::min<int64_t>(H - 1, L - p * H);
        a.write_lower = p == P_last ? 1 : 0;
        a.write_upper = (a.upper > 0 && p * H + a.upper == L) ? 1 : 0;
        a.tiles = M;
        a.nstruct_max = S;
        a.flank_in = p == 0 ? nullptr : fl[(p - 1) & 1].data();
        a.flank_out = fl[p & 1].data();
        a.state = st.data();
        const int64_t ns = (p & 1) ? (periodic ? M : M + 1) : M;
        for (int64_t b = 0; b < ns; ++b) cpu_structure(sch, a, b, work.data(), wr);
    }
}

int main(int argc, char **argv) {
    if (argc != 11) return 2;
    const int scheme = atoi(argv[1]), prec = atoi(argv[2]);
    const int64_t n = atoll(argv[3]);
    const int W = atoi(argv[4]), per = atoi(argv[5]);
    const int64_t steps = atoll(argv[6]);
    const double prm = atof(argv[7]), gamma = atof(argv[8]);
    const int nv = scheme == 0 ? 1 : 3;
    std::vector<double> x((size_t)nv * n);
    FILE *f = fopen(argv[9], "rb");
    if (!f || fread(x.data(), 8, x.size(), f) != x.size()) return 3;
    fclose(f);
    // working layouts as the library's: FP32 rounds, hi/lo splits x = hi + lo
    auto to_f = [&](int planes_lo) {
        std::vector<float> s((size_t)nv * n * (planes_lo ? 2 : 1));
        for (size_t i = 0; i < x.size(); ++i) {
            const float h = (float)x[i];
            s[i] = h;
            if (planes_lo) s[x.size() + i] = (float)(x[i] - (double)h);
        }
        return s;
    };
    EulerParams ep{gamma, gamma - 1.0, prm, 0.5 * prm, (float)gamma, (float)(gamma - 1.0), (float)prm,
                   (float)(0.5 * prm)};
    const float rf = (float)prm, rl = (float)(prm - (double)rf);
    if (prec == 0) {
        if (scheme == 0) run(HostHeatPlain<HostOpsD>{prm}, x, n, W, per, steps);
        else run(HostEuler<HostOpsD, false>{eu_k<HostOpsD>(ep), {}}, x, n, W, per, 4 * steps);
    } else {
        std::vector<float> s = to_f(prec == 2);
        if (scheme == 0 && prec == 1) run(HostHeatPlain<HostOpsF>{rf}, s, n, W, per, steps);
        else if (scheme == 0) run(HostHeatComp{rf, rl}, s, n, W, per, steps);
        else if (prec == 1) run(HostEuler<HostOpsF, false>{eu_k<HostOpsF>(ep), {}}, s, n, W, per, 4 * steps);
        else run(HostEuler<HostOpsF, true>{eu_k<HostOpsF>(ep), {}}, s, n, W, per, 4 * steps);
        for (size_t i = 0; i < x.size(); ++i) x[i] = (double)s[i] + (prec == 2 ? (double)s[x.size() + i] : 0.0);
    }
    f = fopen(argv[10], "wb");
    if (!f || fwrite(x.data(), 8, x.size(), f) != x.size()) return 4;
    fclose(f);
    return 0;
}
