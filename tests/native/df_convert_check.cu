// Host-side check of the integer-pipe FP64 <-> FP32 conversions in
// qbvm_fft.cuh against the hardware casts: split(x) must give
// hi == (float)x and lo == (float)(x - (double)hi), and join(hi, lo) must equal
// (double)hi + (double)lo (the same values the device code computes).
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "qbvm_fft.cuh"

int main() {
    std::mt19937_64 rng(12345);
    long long bad_split = 0, bad_join = 0, n = 0;
    auto check = [&](double x) {
        float hi, lo;
        qbvm::qbvm_split_d(x, &hi, &lo);
        float h0 = (float)x;
        float l0 = (float)(x - (double)h0);
        if (std::memcmp(&hi, &h0, 4) != 0 || std::memcmp(&lo, &l0, 4) != 0) {
            if (bad_split < 5) printf("split mismatch x=%.17g hi=%.9g/%.9g lo=%.9g/%.9g\n", x, hi, h0, lo, l0);
            ++bad_split;
        }
        double j = qbvm::qbvm_join_df(h0, l0);
        double j0 = (double)h0 + (double)l0;
        if (std::memcmp(&j, &j0, 8) != 0) {
            if (bad_join < 5) printf("join mismatch x=%.17g got %.17g want %.17g\n", x, j, j0);
            ++bad_join;
        }
        ++n;
    };
    // random bit patterns over the exponent range an FP32 pair can carry
    for (int i = 0; i < 2000000; ++i) {
        uint64_t m = rng() & 0xFFFFFFFFFFFFFull;
        int e = 1023 - 140 + (int)(rng() % 280);
        uint64_t s = rng() & 1;
        uint64_t b = (s << 63) | ((uint64_t)e << 52) | m;
        double x;
        std::memcpy(&x, &b, 8);
        check(x);
    }
    // rounding ties, carries into a new binade, exact values, zeros
    const double special[] = {0.0, -0.0, 1.0, -1.0, 0.5, 3.0, 1.0 + std::ldexp(1.0, -24), 1.0 + std::ldexp(3.0, -25),
                              std::nextafter(2.0, 1.0), std::ldexp(1.0, 100), std::ldexp(1.0, -100), 1e-30, 1e30,
                              -7.123456789012345e-5, 65504.0, 1.0 - std::ldexp(1.0, -54)};
    for (double x : special) check(x);
    // zero hi with a normal lo, and signed zeros
    const float zs[] = {0.0f, -0.0f};
    for (float z : zs)
        for (float l : {0.0f, -0.0f, 1.5e-3f, -2.25e7f, 3.0e-30f}) {
            double j = qbvm::qbvm_join_df(z, l), j0 = (double)z + (double)l;
            if (std::memcmp(&j, &j0, 8) != 0) {
                printf("zero-hi join mismatch %g %g\n", (double)z, (double)l);
                ++bad_join;
            }
        }
    for (int k = -60; k <= 60; ++k)
        for (int t = 0; t < 64; ++t) check(std::ldexp(1.0 + t * std::ldexp(1.0, -29), k));
    // arbitrary pairs: lo anywhere from ulp(hi)/2 down to far below hi's precision
    std::uniform_real_distribution<double> u(0.5, 1.0);
    for (int i = 0; i < 1000000; ++i) {
        float h = (float)std::ldexp(u(rng) * ((rng() & 1) ? 1 : -1), (int)(rng() % 120) - 60);
        float l = (float)std::ldexp(u(rng) * ((rng() & 1) ? 1 : -1), std::ilogb(h) - 25 - (int)(rng() % 60));
        double j = qbvm::qbvm_join_df(h, l), j0 = (double)h + (double)l;
        if (std::memcmp(&j, &j0, 8) != 0) {
            if (bad_join < 5) printf("pair join mismatch %.9g %.9g: %.17g vs %.17g\n", h, l, j, j0);
            ++bad_join;
        }
        ++n;
    }
    // opposite signs within a binade: exact and heavy cancellation
    for (int i = 0; i < 200000; ++i) {
        float h = (float)std::ldexp(u(rng), (int)(rng() % 120) - 60);
        float l = -(float)std::ldexp(u(rng), std::ilogb(h) - (int)(rng() % 2));
        if (i % 7 == 0) l = -h;
        if (i % 11 == 0) l = -std::nextafter(h, 0.0f);
        if (std::fabs(l) > std::fabs(h)) std::swap(h, l);
        double j = qbvm::qbvm_join_df(h, l), j0 = (double)h + (double)l;
        if (std::memcmp(&j, &j0, 8) != 0) {
            if (bad_join < 5) printf("cancelling join mismatch %.9g %.9g: %.17g vs %.17g\n", h, l, j, j0);
            ++bad_join;
        }
        ++n;
    }
    printf("checked %lld values: split mismatches %lld, join mismatches %lld\n", n, bad_split, bad_join);
    return (bad_split || bad_join) ? 1 : 0;
}
