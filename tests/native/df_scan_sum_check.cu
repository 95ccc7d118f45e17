// Host-side check of the FP64 alpha sweep's double-float spectral sum
// (qbvm_dfsum.cuh): sum over the H even frequencies of Re 1/(d_{2m} + tau
// Lambda) with d_{2m} = 1 - g cos(theta_m) - i g sin(theta_m), g = |omega|^(1/N_t),
// theta_m = pi (4m + 1) / N_t, accumulated as the kernel does (one term per
// frequency, the low word folded every four), against the same sum in long
// double.  Two input sets: a wide one (N_t from 4 to 1024, |omega| from 1e-2
// to 1e8, so Re d and the sum change sign, tau Lambda from 1e-4 to 1e5) and the
// ranges of the 512-instance sweep workload (N_t 32...512, |omega| 1e1...1e6,
// tau Lambda from the lowest mode up by 1e6).
// Prints the largest error relative to the sum of |terms| and to the sum (and
// that of FP64 summation of the same terms), and the largest error of one term
// relative to the larger of |term| and (|Re d| + tau Lambda) / |z|^2, the scale
// FP64's own rounding of Re d + tau Lambda sets.
#include <cmath>
#include <cstdio>
#include <random>

#include "qbvm_dfsum.cuh"

static void split(double x, float& h, float& l) {
    h = (float)x;
    l = (float)(x - (double)h);
}

// One set of 4000 sums: N_t = nt0 << k (k < nk), |omega| = 10^(om0 + om_span u),
// tau Lambda = lam0 10^(lam_span u) (lam0 < 0: (0.1 / (N_t - 1)) pi^2, the
// lowest mode of the unit interval up to T = 0.1).
static void run(const char* name, int nt0, int nk, double om0, double om_span, double lam0, double lam_span) {
    std::mt19937_64 rng(2107);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    double worst_abs = 0.0, worst_rel = 0.0, worst_term = 0.0, worst_f64 = 0.0;
    long long sums = 0, terms = 0;
    for (int trial = 0; trial < 4000; ++trial) {
        const int nt = nt0 << (int)(U(rng) * nk);
        const int H = nt / 2;
        const double om = std::pow(10.0, om0 + om_span * U(rng));
        const double g = std::pow(om, 1.0 / nt);
        const double base = lam0 > 0 ? lam0 : (0.1 / (nt - 1)) * M_PI * M_PI;
        const double lam = base * std::pow(10.0, lam_span * U(rng));
        float lh, ll;
        split(lam, lh, ll);
        float shi = 0.f, slo = 0.f;
        long double ref = 0.0L, mag = 0.0L;
        double s64 = 0.0;
        for (int m0 = 0; m0 < H; m0 += 4) {
            for (int m = m0; m < H && m < m0 + 4; ++m) {
                const double th = M_PI * ((4.0 * m + 1.0) / nt);
                const double re = 1.0 - g * std::cos(th), im = -g * std::sin(th);
                float rh, rl, ih, il;
                split(re, rh, rl);
                split(im, ih, il);
                // the reference takes the values the kernel reads (the table's split
                // of Re d and Im d), so it measures the arithmetic alone
                const long double zr = ((long double)rh + rl) + ((long double)lh + ll);
                const long double zi = (long double)ih + il;
                const long double den = zr * zr + zi * zi, term = zr / den;
                // the same term in FP64 arithmetic, as the FP64 sums compute it
                const double zr64 = ((double)rh + rl) + ((double)lh + ll), zi64 = (double)ih + il;
                s64 += zr64 / (zr64 * zr64 + zi64 * zi64);
                // the term's own scale: FP64 rounds Re d + tau Lambda at 2^-53 of
                // (|Re d| + tau Lambda), an error of that over den in the term
                const long double scale = (fabsl((long double)rh + rl) + ((long double)lh + ll)) / den;
                ref += term;
                mag += fabsl(term);
                float th1 = 0.f, tl1 = 0.f;
                const qbvm::DfSq im2 = qbvm::df_scan_im2(ih, il);
                qbvm::df_scan_term(rh, rl, im2, lh, ll, th1, tl1);
                const long double one = (long double)th1 + tl1;
                const double e = (double)(fabsl(one - term) / fmaxl(fabsl(term), scale));
                if (e > worst_term) worst_term = e;
                ++terms;
                qbvm::df_scan_term(rh, rl, im2, lh, ll, shi, slo);
            }
            qbvm::df_scan_fold(shi, slo);
        }
        const long double got = (long double)shi + slo;
        const double ea = (double)(fabsl(got - ref) / mag);
        const double er = (double)(fabsl(got - ref) / fabsl(ref));
        const double e64 = (double)(fabsl((long double)s64 - ref) / fabsl(ref));
        if (ea > worst_abs) worst_abs = ea;
        if (er > worst_rel) worst_rel = er;
        if (e64 > worst_f64) worst_f64 = e64;
        ++sums;
    }
    printf("[%s] sums %lld terms %lld\n", name, sums, terms);
    printf("[%s] max |err| / sum|terms| %.3e\n", name, worst_abs);
    printf("[%s] max |err| / |sum| %.3e\n", name, worst_rel);
    printf("[%s] max |err| / |sum| in FP64 %.3e\n", name, worst_f64);
    printf("[%s] max term err / max(|term|, (|Re d| + tau Lambda) / |z|^2) %.3e\n", name, worst_term);
}

int main() {
    run("wide", 4, 9, -2.0, 10.0, 1e-4, 9.0);        // N_t 4..1024, |omega| 1e-2..1e8, tau Lambda 1e-4..1e5
    run("sweep", 32, 5, 1.0, 5.0, -1.0, 6.0);        // N_t 32..512, |omega| 1e1..1e6, tau Lambda from the lowest mode
    return 0;
}
