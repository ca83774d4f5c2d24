// Host driver for the double-FP32 primitives of csrc/df.cuh (built and run
// by tests/test_df_host.py on the CPU; no GPU).  It draws float / df
// operands over a wide exponent range from a fixed xorshift stream and
// prints operands and results as C99 hex floats; the Python side checks
// them with exact rational arithmetic.
#include <cstdint>
#include <cstdio>

#include "df.cuh"

using namespace shtg;

static uint64_t g_state = 0x9E3779B97F4A7C15ull;
static uint64_t next_u64() {   // xorshift64*
    g_state ^= g_state >> 12;
    g_state ^= g_state << 25;
    g_state ^= g_state >> 27;
    return g_state * 0x2545F4914F6CDD1Dull;
}
static double unit() { return (double)(next_u64() >> 11) * (1.0 / 9007199254740992.0); }
// |x| in [2^-40, 2^40], random sign
static double wide() {
    const double mant = 1.0 + unit();
    const int ex = (int)(next_u64() % 81) - 40;
    double x = mant;
    for (int i = 0; i < (ex < 0 ? -ex : ex); ++i) x = ex < 0 ? x * 0.5 : x * 2.0;
    return (next_u64() & 1) ? -x : x;
}
// |x| in [0.5, 2), random sign (operands of similar size: cancellation)
static double near1() {
    const double x = 0.5 + 1.5 * unit();
    return (next_u64() & 1) ? -x : x;
}

int main() {
    const int N = 4000;
    for (int i = 0; i < N; ++i) {
        const float a = (float)wide(), b = (float)wide();
        float e;
        const float s = two_sum(a, b, e);
        std::printf("two_sum %a %a %a %a\n", a, b, s, e);
        const float p = two_prod(a, b, e);
        std::printf("two_prod %a %a %a %a\n", a, b, p, e);
        const float big = fabsf(a) >= fabsf(b) ? a : b, small = fabsf(a) >= fabsf(b) ? b : a;
        const float fs = fast_two_sum(big, small, e);
        std::printf("fast_two_sum %a %a %a %a\n", big, small, fs, e);
    }
    for (int i = 0; i < N; ++i) {
        const double x = (i & 1) ? wide() : near1(), y = (i & 2) ? wide() : near1();
        const df dx = df_from(x), dy = df_from(y);
        std::printf("from %a %a %a\n", x, dx.hi, dx.lo);
        const df s = df_add(dx, dy);
        std::printf("add %a %a %a %a %a %a\n", dx.hi, dx.lo, dy.hi, dy.lo, s.hi, s.lo);
        const df m = df_mul(dx, dy);
        std::printf("mul %a %a %a %a %a %a\n", dx.hi, dx.lo, dy.hi, dy.lo, m.hi, m.lo);
        std::printf("to %a %a %a\n", dx.hi, dx.lo, df_to(dx));
    }
    // dot products as the Legendre kernels accumulate them: df_fma into a
    // running sum, renormalised every 32 terms
    for (int t = 0; t < 200; ++t) {
        const int n = 1 + (int)(next_u64() % 512);
        dfacc acc;
        df_acc_zero(acc);
        std::printf("dot %d", n);
        for (int k = 0; k < n; ++k) {
            const df u = df_from(near1()), v = df_from(wide() * 1e-3);
            df_fma(acc, u, v);
            if ((k & 31) == 31) df_acc_norm(acc);
            std::printf(" %a %a %a %a", u.hi, u.lo, v.hi, v.lo);
        }
        df_acc_norm(acc);
        std::printf(" %a %a\n", acc.hi, acc.lo);
    }
    return 0;
}
