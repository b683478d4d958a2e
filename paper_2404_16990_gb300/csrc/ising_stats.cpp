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

#include <algorithm>
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


// ---------------------------------------------------------------------------
// Random-stream battery (the paper's generator checks, supplementary PRNG
// tests: the NIST SP 800-22 bit tests, then floats for uniformity in 100
// bins, lag-1 independence, and the bits "float >= median").
// ---------------------------------------------------------------------------

// Regularised upper incomplete gamma Q(a, x): the power series of the lower
// function for x < a + 1, else Legendre's continued fraction evaluated by the
// modified Lentz method (as in Press et al., Numerical Recipes, section 6.2).
double gamma_q(double a, double x) {
    if (!(x > 0.0)) return 1.0;
    const double lg = std::lgamma(a);
    if (x < a + 1.0) {
        double term = 1.0 / a, sum = term;
        for (int k = 1; k < 100000; ++k) {
            term *= x / (a + k);
            sum += term;
            if (std::fabs(term) < std::fabs(sum) * 1e-17) break;
        }
        const double P = sum * std::exp(-x + a * std::log(x) - lg);
        return 1.0 - P;
    }
    const double tiny = 1e-300;
    double b = x + 1.0 - a, c = 1.0 / tiny, d = 1.0 / b, h = d;
    for (int i = 1; i < 100000; ++i) {
        const double an = -i * (i - a);
        b += 2.0;
        d = an * d + b;
        if (std::fabs(d) < tiny) d = tiny;
        c = b + an / c;
        if (std::fabs(c) < tiny) c = tiny;
        d = 1.0 / d;
        const double del = d * c;
        h *= del;
        if (std::fabs(del - 1.0) < 1e-17) break;
    }
    return std::exp(-x + a * std::log(x) - lg) * h;
}

double phi(double x) { return 0.5 * std::erfc(-x / std::sqrt(2.0)); }

void t_frequency(const std::vector<uint8_t>& b, double* p, double* st) {
    const int64_t n = (int64_t)b.size();
    int64_t ones = 0;
    for (uint8_t v : b) ones += v;
    const double S = 2.0 * (double)ones - (double)n;
    *st = S;
    *p = std::erfc(std::fabs(S) / std::sqrt(2.0 * (double)n));
}

void t_block_frequency(const std::vector<uint8_t>& b, int M, double* p, double* st) {
    const int64_t N = (int64_t)b.size() / M;
    double chi2 = 0.0;
    for (int64_t j = 0; j < N; ++j) {
        int64_t ones = 0;
        for (int i = 0; i < M; ++i) ones += b[(size_t)(j * M + i)];
        const double d = (double)ones / M - 0.5;
        chi2 += d * d;
    }
    chi2 *= 4.0 * M;
    *st = chi2;
    *p = gamma_q((double)N / 2.0, chi2 / 2.0);
}

void t_runs(const std::vector<uint8_t>& b, double* p, double* st) {
    const int64_t n = (int64_t)b.size();
    int64_t ones = 0;
    for (uint8_t v : b) ones += v;
    const double pi = (double)ones / (double)n;
    if (std::fabs(pi - 0.5) >= 2.0 / std::sqrt((double)n)) {
        *p = 0.0;
        *st = NAN;
        return;
    }
    int64_t V = 1;
    for (int64_t i = 0; i + 1 < n; ++i) V += b[(size_t)i] != b[(size_t)i + 1];
    const double num = std::fabs((double)V - 2.0 * (double)n * pi * (1.0 - pi));
    const double den = 2.0 * std::sqrt(2.0 * (double)n) * pi * (1.0 - pi);
    *st = (double)V;
    *p = std::erfc(num / den);
}

// P(longest run of ones <= k) in M fair bits: count of strings with no run
// longer than k, f(m) = 2^m (m <= k), f(m) = sum_{j=0..k} f(m-1-j), over 2^M,
// carried as probabilities (f(m) / 2^m) to stay in range
double prob_longest_at_most(int M, int k) {
    std::vector<double> q((size_t)M + 1);
    for (int m = 0; m <= M; ++m) {
        if (m <= k) {
            q[(size_t)m] = 1.0;
        } else {
            double s = 0.0;
            for (int j = 0; j <= k; ++j) s += q[(size_t)(m - 1 - j)] * std::ldexp(1.0, -(1 + j));
            q[(size_t)m] = s;
        }
    }
    return q[(size_t)M];
}

void t_longest_run(const std::vector<uint8_t>& b, double* p, double* st) {
    const int M = 128, lo = 4, hi = 9, K = hi - lo;
    const int64_t N = (int64_t)b.size() / M;
    std::vector<double> counts((size_t)K + 1, 0.0);
    for (int64_t j = 0; j < N; ++j) {
        int best = 0, cur = 0;
        for (int i = 0; i < M; ++i) {
            cur = b[(size_t)(j * M + i)] ? cur + 1 : 0;
            best = std::max(best, cur);
        }
        counts[(size_t)(std::min(std::max(best, lo), hi) - lo)] += 1.0;
    }
    std::vector<double> cum((size_t)K);
    for (int k = lo; k < hi; ++k) cum[(size_t)(k - lo)] = prob_longest_at_most(M, k);
    double chi2 = 0.0;
    for (int c = 0; c <= K; ++c) {
        const double pc = (c == 0) ? cum[0] : (c == K ? 1.0 - cum[(size_t)K - 1] : cum[(size_t)c] - cum[(size_t)c - 1]);
        const double e = (double)N * pc;
        chi2 += (counts[(size_t)c] - e) * (counts[(size_t)c] - e) / e;
    }
    *st = chi2;
    *p = gamma_q(K / 2.0, chi2 / 2.0);
}

void t_spectral(const std::vector<uint8_t>& b, double* p, double* st) {
    int64_t n = 1;
    while (n * 2 <= (int64_t)b.size() && n * 2 <= (int64_t)ISING_PRNG_SPECTRAL_MAX_BITS) n *= 2;
    std::vector<std::complex<double>> a((size_t)n);
    for (int64_t i = 0; i < n; ++i) a[(size_t)i] = std::complex<double>(2.0 * b[(size_t)i] - 1.0, 0.0);
    fft(a, false);
    const double T = std::sqrt(std::log(1.0 / 0.05) * (double)n);
    int64_t N1 = 0;
    for (int64_t k = 0; k < n / 2; ++k) N1 += std::abs(a[(size_t)k]) < T;
    const double N0 = 0.95 * (double)n / 2.0;
    const double d = ((double)N1 - N0) / std::sqrt((double)n * 0.95 * 0.05 / 4.0);
    *st = d;
    *p = std::erfc(std::fabs(d) / std::sqrt(2.0));
}

void t_cusum(const std::vector<uint8_t>& b, bool reverse, double* p, double* st) {
    const int64_t n = (int64_t)b.size();
    int64_t S = 0, z = 0;
    for (int64_t i = 0; i < n; ++i) {
        S += b[(size_t)(reverse ? n - 1 - i : i)] ? 1 : -1;
        z = std::max(z, S < 0 ? -S : S);
    }
    *st = (double)z;
    if (z == 0) {
        *p = 0.0;
        return;
    }
    const double nz = (double)n / (double)z, sq = std::sqrt((double)n), zd = (double)z;
    double s1 = 0.0, s2 = 0.0;
    for (int64_t k = (int64_t)std::floor((-nz + 1.0) / 4.0); k <= (int64_t)std::floor((nz - 1.0) / 4.0); ++k)
        s1 += phi((4.0 * k + 1.0) * zd / sq) - phi((4.0 * k - 1.0) * zd / sq);
    for (int64_t k = (int64_t)std::floor((-nz - 3.0) / 4.0); k <= (int64_t)std::floor((nz - 1.0) / 4.0); ++k)
        s2 += phi((4.0 * k + 3.0) * zd / sq) - phi((4.0 * k + 1.0) * zd / sq);
    *p = 1.0 - s1 + s2;
}

void t_float_uniformity(const std::vector<double>& f, double* p, double* st) {
    const int bins = 100;
    std::vector<double> c((size_t)bins, 0.0);
    for (double v : f) c[(size_t)std::min((int)(v * bins), bins - 1)] += 1.0;
    const double e = (double)f.size() / bins;
    double chi2 = 0.0;
    for (double v : c) chi2 += (v - e) * (v - e) / e;
    *st = chi2;
    *p = gamma_q((bins - 1) / 2.0, chi2 / 2.0);
}

void t_float_pairs(const std::vector<double>& f, double* p, double* st) {
    const int bins = 10;
    const size_t n = f.size() / 2;
    std::vector<double> c((size_t)bins * bins, 0.0);
    for (size_t i = 0; i < n; ++i) {
        const int x = std::min((int)(f[2 * i] * bins), bins - 1), y = std::min((int)(f[2 * i + 1] * bins), bins - 1);
        c[(size_t)(x * bins + y)] += 1.0;
    }
    const double e = (double)n / (bins * bins);
    double chi2 = 0.0;
    for (double v : c) chi2 += (v - e) * (v - e) / e;
    *st = chi2;
    *p = gamma_q((bins * bins - 1) / 2.0, chi2 / 2.0);
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

int ising_prng_battery(const uint32_t* words, int64_t n_words, double* pvalues, double* statistics) {
    if (!words || !pvalues) return ising::set_last_error(ISING_EINVAL, "words or pvalues is NULL");
    if (n_words < 4096) return ising::set_last_error(ISING_EINVAL, "the battery needs at least 4096 words");
    if (n_words > ((int64_t)1 << 30)) return ising::set_last_error(ISING_EINVAL, "at most 2^30 words");
    const int64_t n = n_words * 32;
    std::vector<uint8_t> b((size_t)n);
    for (int64_t i = 0; i < n; ++i) b[(size_t)i] = (uint8_t)((words[i >> 5] >> (31 - (i & 31))) & 1u);
    std::vector<double> f((size_t)n_words);
    for (int64_t i = 0; i < n_words; ++i) f[(size_t)i] = (double)(words[i] & 0x7FFFFFu) / (double)(1u << 23);
    // bits "float >= median" (median as the mean of the two middle values for
    // an even count)
    std::vector<double> sorted = f;
    const size_t h = sorted.size() / 2;
    std::nth_element(sorted.begin(), sorted.begin() + (std::ptrdiff_t)h, sorted.end());
    double med = sorted[h];
    if (sorted.size() % 2 == 0) {
        const double lower = *std::max_element(sorted.begin(), sorted.begin() + (std::ptrdiff_t)h);
        med = 0.5 * (lower + med);
    }
    std::vector<uint8_t> mb(f.size());
    for (size_t i = 0; i < f.size(); ++i) mb[i] = f[i] >= med;
    double st[ISING_PRNG_TESTS];
    t_frequency(b, &pvalues[0], &st[0]);
    t_block_frequency(b, 128, &pvalues[1], &st[1]);
    t_runs(b, &pvalues[2], &st[2]);
    t_longest_run(b, &pvalues[3], &st[3]);
    t_spectral(b, &pvalues[4], &st[4]);
    t_cusum(b, false, &pvalues[5], &st[5]);
    t_cusum(b, true, &pvalues[6], &st[6]);
    t_float_uniformity(f, &pvalues[7], &st[7]);
    t_float_pairs(f, &pvalues[8], &st[8]);
    t_runs(mb, &pvalues[9], &st[9]);
    t_longest_run(mb, &pvalues[10], &st[10]);
    if (statistics)
        for (int i = 0; i < ISING_PRNG_TESTS; ++i) statistics[i] = st[i];
    return ISING_OK;
}

}  // extern "C"
