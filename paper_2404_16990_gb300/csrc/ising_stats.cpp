// ising_stats.cpp -- host statistics of Monte Carlo time series: integrated
// autocorrelation time with the automatic window of Madras and Sokal (J. Stat.
// Phys. 50, 109 (1988); A. D. Sokal, "Monte Carlo methods in statistical
// mechanics", 1997), and the Binder cumulant from FP64 moment sums.
//
// The paper averages |M| every 10^4-2*10^4 sweeps and discards the
// non-equilibrated part (Section 3.1); these routines give the error bars and
// effective sample counts that such averages need.
#include "../../include/ising.h"
#include "ising_internal.h"

#include <cmath>
#include <cstdint>

extern "C" {

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
    for (int64_t lag = 1; lag <= max_lag; ++lag) {
        double s = 0.0;
        for (int64_t i = 0; i + lag < n; ++i) s += (x[i] - mean) * (x[i + lag] - mean);
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
