// ising_stats.cpp -- host statistics of Monte Carlo time series: integrated
// autocorrelation time with the automatic window of Madras and Sokal (J. Stat.
// Phys. 50, 109 (1988); A. D. Sokal, "Monte Carlo methods in statistical
// mechanics", 1997), the Binder cumulant from FP64 moment sums, and the
// statistical inefficiency with automatic equilibration detection of Chodera
// (J. Chem. Theory Comput. 12, 1799 (2016)).
//
// The paper averages |M| every 10^4-2*10^4 sweeps and discards the
// non-equilibrated part with Chodera's method (Section 3.1); these routines
// give the equilibrated start, error bars and effective sample counts that
// such averages need.
#include "../../include/ising.h"
#include "ising_internal.h"

#include <cmath>
#include <complex>
#include <cstdint>
#include <vector>

namespace {

// In-place iterative radix-2 FFT (Cooley-Tukey); n is a power of two.
void fft(std::vector<std::complex<double>>& a, bool inverse) {
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const double ang = 2.0 * M_PI / (double)len * (inverse ? 1.0 : -1.0);
        const std::complex<double> wl(std::cos(ang), std::sin(ang));
        for (size_t i = 0; i < n; i += len) {
            std::complex<double> w(1.0, 0.0);
            for (size_t k = 0; k < len / 2; ++k) {
                const std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
                w *= wl;
            }
        }
    }
    if (inverse)
        for (auto& x : a) x /= (double)n;
}

// sum_{i} d[i] d[i + lag] for lag = 0 .. n-1 (d = x - mean), by FFT.
std::vector<double> autocov_sums(const double* x, int64_t n, double mean) {
    size_t m = 1;
    while (m < 2 * (size_t)n) m <<= 1;
    std::vector<std::complex<double>> a(m, 0.0);
    for (int64_t i = 0; i < n; ++i) a[i] = x[i] - mean;
    fft(a, false);
    for (auto& v : a) v = std::complex<double>(std::norm(v), 0.0);
    fft(a, true);
    std::vector<double> out((size_t)n);
    for (int64_t i = 0; i < n; ++i) out[i] = a[i].real();
    return out;
}

// Statistical inefficiency g = 1 + 2 sum_{t>=1} (1 - t/n) C(t) of x[0..n-1],
// C(t) = [sum_{i<n-t} d_i d_{i+t} / (n - t)] / [sum_i d_i^2 / n] about the
// series' own mean, the sum stopping before the first lag with C(t) <= 0;
// at least 1.  Lag sums by FFT on long series, one lag at a time otherwise.
double stat_ineff(const double* x, int64_t n) {
    double mean = 0.0;
    for (int64_t i = 0; i < n; ++i) mean += x[i];
    mean /= (double)n;
    double var = 0.0;
    for (int64_t i = 0; i < n; ++i) var += (x[i] - mean) * (x[i] - mean);
    var /= (double)n;
    if (!(var > 0.0)) return 1.0;
    std::vector<double> sums;
    if (n >= 4096) sums = autocov_sums(x, n, mean);
    double tau = 0.0;
    for (int64_t t = 1; t < n; ++t) {
        double s = 0.0;
        if (!sums.empty()) {
            s = sums[(size_t)t];
        } else {
            for (int64_t i = 0; i + t < n; ++i) s += (x[i] - mean) * (x[i + t] - mean);
        }
        const double C = s / ((double)(n - t) * var);
        if (!(C > 0.0)) break;
        tau += (1.0 - (double)t / (double)n) * C;
    }
    const double g = 1.0 + 2.0 * tau;
    return g < 1.0 ? 1.0 : g;
}

}  // namespace

extern "C" {

int ising_stat_inefficiency(const double* x, int64_t n, double* g) {
    if (!x || !g) return ising::set_last_error(ISING_EINVAL, "x or g is NULL");
    if (n < 2) return ising::set_last_error(ISING_EINVAL, "series needs at least 2 points");
    *g = stat_ineff(x, n);
    return ISING_OK;
}

int ising_equilibration(const double* x, int64_t n, int64_t stride, int64_t* t0, double* g, double* n_eff) {
    if (!x || !t0) return ising::set_last_error(ISING_EINVAL, "x or t0 is NULL");
    if (n < 2) return ising::set_last_error(ISING_EINVAL, "series needs at least 2 points");
    if (stride < 0) return ising::set_last_error(ISING_EINVAL, "stride must be >= 0");
    if (stride == 0) stride = n / 256 > 1 ? n / 256 : 1;
    double best_n = -1.0, best_g = 1.0;
    int64_t best_t = 0;
    for (int64_t s = 0; s <= n - 2; s += stride) {
        const double gs = stat_ineff(x + s, n - s);
        const double ns = (double)(n - s) / gs;
        if (ns > best_n) {
            best_n = ns;
            best_g = gs;
            best_t = s;
        }
    }
    *t0 = best_t;
    if (g) *g = best_g;
    if (n_eff) *n_eff = best_n;
    return ISING_OK;
}

int ising_tau_int(const double* x, int64_t n, double c, double* tau, double* tau_err, int64_t* window) {
    if (!x || !tau) return ising::set_last_error(ISING_EINVAL, "x or tau is NULL");
    if (n < 2) return ising::set_last_error(ISING_EINVAL, "series needs at least 2 points");
    if (!(c > 0.0)) return ising::set_last_error(ISING_EINVAL, "window factor c must be positive");
    double mean = 0.0;
    for (int64_t i = 0; i < n; ++i) mean += x[i];
    mean /= (double)n;
    double c0 = 0.0;
    for (int64_t i = 0; i < n; ++i) c0 += (x[i] - mean) * (x[i] - mean);
    c0 /= (double)n;
    if (!(c0 > 0.0)) {  // constant series: no fluctuations, tau = 1/2 by convention
        *tau = 0.5;
        if (tau_err) *tau_err = 0.0;
        if (window) *window = 0;
        return ISING_OK;
    }
    double t = 0.5;
    int64_t M = 0;
    const int64_t max_lag = n / 2;
    // autocovariance sums for every lag at once (FFT) on long series, one lag
    // at a time on short ones
    std::vector<double> sums;
    if (n >= 4096) sums = autocov_sums(x, n, mean);
    for (int64_t lag = 1; lag <= max_lag; ++lag) {
        double s = 0.0;
        if (!sums.empty()) {
            s = sums[(size_t)lag];
        } else {
            for (int64_t i = 0; i + lag < n; ++i) s += (x[i] - mean) * (x[i + lag] - mean);
        }
        const double rho = s / ((double)n * c0);
        t += rho;
        M = lag;
        if ((double)lag >= c * t) break;
    }
    *tau = t;
    if (tau_err) *tau_err = t * std::sqrt(2.0 * (2.0 * (double)M + 1.0) / (double)n);
    if (window) *window = M;
    return ISING_OK;
}

int ising_binder(const double* moments, int n_sims, double* U) {
    if (n_sims < 0 || (n_sims > 0 && (!moments || !U)))
        return ising::set_last_error(ISING_EINVAL, "invalid arguments");
    for (int i = 0; i < n_sims; ++i) {
        const double* m = moments + 6 * (size_t)i;
        const double cnt = m[0];
        if (!(cnt > 0.0)) { U[i] = NAN; continue; }
        const double m2 = m[2] / cnt, m4 = m[3] / cnt;
        U[i] = (m2 > 0.0) ? 1.0 - m4 / (3.0 * m2 * m2) : NAN;
    }
    return ISING_OK;
}

}  // extern "C"
