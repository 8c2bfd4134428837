// Host-only harness for tests/test_fp64_soft.py: the integer-pipe FP64 heat
// update (csrc/fp64_soft.cuh, compiled here as host code) against the host's own
// IEEE 754 binary64 arithmetic, fma(r, fma(-2, u, a + b), u) with std::fma and
// no contraction. Every case the integer path accepts must give the same bits.
//
// usage: fp64_soft_check seed cases_per_family
// prints one line per family: name cases fast mismatches; exit 1 on any mismatch.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "fp64_soft.cuh"

using namespace sw;

static std::mt19937_64 rng;
static long g_bad = 0;

struct Count {
    long cases = 0, fast = 0, bad = 0;
};

static double ieee(double r, double a, double u, double b) { return std::fma(r, std::fma(-2.0, u, a + b), u); }

static void check(Count &c, double r, double a, double u, double b) {
    const soft64::HeatR h = soft64::make_heat_r(r);
    bool ok = true;
    const uint64_t got = soft64::heat_update(h, soft64::bits(a), soft64::bits(u), soft64::bits(b), ok);
    ++c.cases;
    if (!(ok && h.usable)) return;
    ++c.fast;
    const double want = ieee(r, a, u, b);
    if (got != soft64::bits(want)) {
        if (g_bad++ < 8)
            std::printf("mismatch r=%a a=%a u=%a b=%a: %a, IEEE %a\n", r, a, u, b, soft64::value(got), want);
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
    std::uniform_real_distribution<double> ur(0.01, 0.5);
    {   // neighbours close to u at every relative scale
        Count c;
        for (long i = 0; i < N; ++i) {
            const double u = rexp(1000, 1040);
            const int sc = (int)(rng() % 50);
            check(c, ur(rng), near(u, sc), u, near(u, sc));
        }
        report("smooth", c);
    }
    {   // one neighbour 2^0 .. 2^-9 of u (across the low edge of the exponent window), the
        // other about 2u - a, so that the second difference stays small
        Count c;
        for (long i = 0; i < N; ++i) {
            const double u = rexp(1020, 1026);
            const double a = near(std::ldexp(u, -(int)(rng() % 10)), 2);
            const double b = near(2.0 * u - a, 20 + (int)(rng() % 30));
            if (rng() & 1) check(c, ur(rng), a, u, b);
            else check(c, ur(rng), b, u, a);
        }
        report("window", c);
    }
    {   // exact ties in the last rounding: r = 2^-j and r d = (K + 1/2) ulp(u)
        Count c;
        for (long i = 0; i < N; ++i) {
            const int j = 1 + (int)(rng() % 6);
            const double u = std::fabs(rexp(1023, 1023)) * ((rng() & 1) ? 1 : -1);
            const double ulp = std::ldexp(1.0, std::ilogb(u) - 52);
            const uint64_t K = rng() >> 34;
            double dd = std::ldexp((double)(2 * K + 1), j - 1) * ulp;
            if (rng() & 1) dd = -dd;
            check(c, std::ldexp(1.0, -j), u + dd, u, u);  // a + b = 2u + dd exactly
        }
        report("ties", c);
    }
    {   // u at the edges of its binade, so that u + r d may leave it
        Count c;
        for (long i = 0; i < N; ++i) {
            const uint64_t frac = (rng() & 1) ? rng() % 1024 : soft64::kFrac - rng() % 1024;
            const double u = soft64::value(((uint64_t)(1021 + rng() % 5) << 52) | frac | (rng() & soft64::kSign));
            const int sc = 20 + (int)(rng() % 30);
            check(c, ur(rng), near(u, sc), u, near(u, sc));
        }
        report("binade", c);
    }
    {   // r with few significant bits (the product's low bits vanish) and across its range
        Count c;
        for (long i = 0; i < N; ++i) {
            const double r = std::ldexp((double)(1 + rng() % 16), -(int)(rng() % 30) - 4);
            const double u = rexp(1010, 1030);
            const int sc = (int)(rng() % 40);
            check(c, r, near(u, sc), u, near(u, sc));
        }
        report("r_bits", c);
    }
    {   // anything: zeros, subnormals, infinities, NaNs, extreme exponents, mixed signs
        Count c;
        for (long i = 0; i < N; ++i) check(c, ur(rng), soft64::value(rng()), soft64::value(rng()), soft64::value(rng()));
        for (long i = 0; i < N; ++i) {
            const double u = rexp(1, 80);
            check(c, ur(rng), near(u, 3), u, near(u, 3));
        }
        for (long i = 0; i < N; ++i) {
            const double u = rexp(2030, 2046);
            check(c, ur(rng), near(u, 3), u, near(u, 3));
        }
        for (long i = 0; i < N; ++i) {
            const double u = rexp(1023, 1023);
            check(c, ur(rng), 0.0, u, (rng() & 1) ? -u : u);
        }
        report("special", c);
    }
    {   // the heat run itself: a periodic field of 32 modes, 400 steps, both paths
        Count c;
        const int n = 4096;
        const double r = 0.3137;
        const soft64::HeatR h = soft64::make_heat_r(r);
        std::vector<double> x(n), y(n);
        for (int j = 0; j < n; ++j) {
            double t = 0;
            for (int m = 1; m <= 32; ++m) t += std::sin(2 * M_PI * (1 + (m * 37) % 64) * j / n + m) * (((m * 13) % 7) - 3) / 3.0;
            x[j] = t;
        }
        for (int step = 0; step < 400; ++step) {
            for (int j = 0; j < n; ++j) {
                const double a = x[(j + n - 1) % n], u = x[j], b = x[(j + 1) % n];
                const double want = ieee(r, a, u, b);
                bool ok = true;
                const uint64_t got = soft64::heat_update(h, soft64::bits(a), soft64::bits(u), soft64::bits(b), ok);
                ++c.cases;
                if (ok) {
                    ++c.fast;
                    if (got != soft64::bits(want)) ++c.bad, ++g_bad;
                }
                y[j] = want;
            }
            std::swap(x, y);
        }
        report("heat_run", c);
    }
    return g_bad ? 1 : 0;
}
