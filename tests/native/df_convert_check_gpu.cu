// Device-side check of the FP64 <-> double-float conversions in qbvm_fft.cuh:
// qbvm_join_df_dadd (bit-built widenings + one FP64 add) and qbvm_join_df
// (integer pipes) must both equal the hardware (double)hi + (double)lo, and
// qbvm_split_d must give hi = (float)x and lo = (float)(x - (double)hi), bit
// for bit, on random and special operands (zeros, subnormals, infinities,
// NaN, unnormalised pairs).
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <limits>
#include <random>
#include <vector>

#include "qbvm_fft.cuh"

__global__ void k_check(const float2* pairs, const double* xs, long long n, double* j_dadd, double* j_int,
                        double* j_hw, float2* sp, float2* sp_hw) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 p = pairs[i];
    j_dadd[i] = qbvm::qbvm_join_df_dadd(p.x, p.y);
    j_int[i] = qbvm::qbvm_join_df(p.x, p.y);
    j_hw[i] = __dadd_rn((double)p.x, (double)p.y);
    float h, l;
    qbvm::qbvm_split_d(xs[i], &h, &l);
    sp[i] = make_float2(h, l);
    const float h0 = (float)xs[i];
    sp_hw[i] = make_float2(h0, (float)(xs[i] - (double)h0));
}

static bool same_bits(double a, double b) {
    if (std::isnan(a) && std::isnan(b)) return true;
    return std::memcmp(&a, &b, 8) == 0;
}
static bool same_bits(float a, float b) {
    if (std::isnan(a) && std::isnan(b)) return true;
    return std::memcmp(&a, &b, 4) == 0;
}

int main() {
    std::mt19937_64 rng(2024);
    std::vector<float2> pairs;
    std::vector<double> xs;
    std::uniform_real_distribution<double> u(0.5, 1.0);
    for (int i = 0; i < 1 << 20; ++i) {
        // a pair from a random double (normalised), and a random pair
        uint64_t b = ((rng() & 1) << 63) | ((uint64_t)(1023 - 140 + (int)(rng() % 280)) << 52) |
                     (rng() & 0xFFFFFFFFFFFFFull);
        double x;
        std::memcpy(&x, &b, 8);
        const float h = (float)x;
        pairs.push_back(make_float2(h, (float)(x - (double)h)));
        xs.push_back(x);
        const float h2 = (float)std::ldexp(u(rng) * ((rng() & 1) ? 1 : -1), (int)(rng() % 240) - 120);
        const float l2 = (float)std::ldexp(u(rng) * ((rng() & 1) ? 1 : -1), std::ilogb(h2) - (int)(rng() % 80));
        pairs.push_back(make_float2(h2, l2));
        xs.push_back(std::ldexp(u(rng), (int)(rng() % 2000) - 1000));
    }
    const float inf = std::numeric_limits<float>::infinity(), nan = std::numeric_limits<float>::quiet_NaN();
    const float sub = std::ldexp(1.0f, -140), fmin = std::numeric_limits<float>::min();
    const float sp_vals[] = {0.0f, -0.0f, 1.0f, -1.0f, sub, -sub, fmin, 3.0e38f, -3.0e38f, inf, -inf, nan, 1.5e-3f};
    for (float a : sp_vals)
        for (float c : sp_vals) {
            pairs.push_back(make_float2(a, c));
            xs.push_back((double)a * 1.000000123);
        }
    const double dsp[] = {0.0, -0.0, 1e-300, -1e300, std::ldexp(1.0, -149), std::ldexp(1.0, -150), 3.5e38,
                          std::numeric_limits<double>::infinity(), std::numeric_limits<double>::quiet_NaN()};
    for (double x : dsp) {
        pairs.push_back(make_float2(1.0f, 0.0f));
        xs.push_back(x);
    }
    const long long n = (long long)pairs.size();
    float2 *dp, *dsp2, *dsh;
    double *dx, *ja, *ji, *jh;
    if (cudaMalloc(&dp, n * sizeof(float2)) || cudaMalloc(&dx, n * 8) || cudaMalloc(&ja, n * 8) ||
        cudaMalloc(&ji, n * 8) || cudaMalloc(&jh, n * 8) || cudaMalloc(&dsp2, n * sizeof(float2)) ||
        cudaMalloc(&dsh, n * sizeof(float2))) {
        printf("allocation failed\n");
        return 2;
    }
    cudaMemcpy(dp, pairs.data(), n * sizeof(float2), cudaMemcpyHostToDevice);
    cudaMemcpy(dx, xs.data(), n * 8, cudaMemcpyHostToDevice);
    k_check<<<(unsigned)((n + 255) / 256), 256>>>(dp, dx, n, ja, ji, jh, dsp2, dsh);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        printf("kernel failed\n");
        return 2;
    }
    std::vector<double> a(n), b(n), c(n);
    std::vector<float2> s(n), s0(n);
    cudaMemcpy(a.data(), ja, n * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(b.data(), ji, n * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(c.data(), jh, n * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(s.data(), dsp2, n * sizeof(float2), cudaMemcpyDeviceToHost);
    cudaMemcpy(s0.data(), dsh, n * sizeof(float2), cudaMemcpyDeviceToHost);
    long long bad_dadd = 0, bad_int = 0, bad_split = 0;
    for (long long i = 0; i < n; ++i) {
        if (!same_bits(a[i], c[i])) {
            if (bad_dadd < 5) printf("dadd join %.9g %.9g: %.17g vs %.17g\n", pairs[i].x, pairs[i].y, a[i], c[i]);
            ++bad_dadd;
        }
        if (!same_bits(b[i], c[i])) {
            if (bad_int < 5) printf("int join %.9g %.9g: %.17g vs %.17g\n", pairs[i].x, pairs[i].y, b[i], c[i]);
            ++bad_int;
        }
        if (!same_bits(s[i].x, s0[i].x) || !same_bits(s[i].y, s0[i].y)) {
            if (bad_split < 5) printf("split %.17g: %.9g %.9g vs %.9g %.9g\n", xs[i], s[i].x, s[i].y, s0[i].x, s0[i].y);
            ++bad_split;
        }
    }
    printf("checked %lld: dadd-join mismatches %lld, int-join mismatches %lld, split mismatches %lld\n", n, bad_dadd,
           bad_int, bad_split);
    return (bad_dadd || bad_int || bad_split) ? 1 : 0;
}
