// Host-side analysis of multicanonical data (Sec. 3): reweighting to
// canonical temperatures, the multi-histogram combination of several
// iterations' histograms into one ln Omega, the Ising map of Eq. 5 and the
// infinite-volume droplet fraction of Biskup et al. as the paper states it
// (Eqs. 8-10).  Double precision, no device work: the inputs are a few
// hundred bins.

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <limits>
#include <vector>

#include "mucal.h"
#include "mucal_internal.h"

namespace {

int bad(const char *fmt, ...)
{
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    mucal::set_init_error(buf);
    return MUCAL_ERR_INVALID_ARG;
}

// f(lambda) = lambda^((d-1)/d) + Delta (1 - lambda)^2, the bracket of Eq. 9.
double droplet_free_energy(int d, double Delta, double lambda)
{
    const double a = (double)(d - 1) / (double)d;
    const double u = 1.0 - lambda;
    return std::pow(lambda, a) + Delta * u * u;
}

}  // namespace

extern "C" {

int mucal_reweight(const int64_t *H, const double *lnW, int32_t n_bins, int32_t e_lo,
                   const double *beta, int32_t n_beta, const double *obs, int32_t n_obs,
                   double *mean_E, double *mean_E2, double *obs_out)
{
    if (!H || !lnW) return bad("H and lnW must not be NULL");
    if (n_bins < 1) return bad("n_bins must be >= 1");
    if (n_beta < 0 || n_obs < 0) return bad("n_beta and n_obs must be >= 0");
    if (n_beta > 0 && !beta) return bad("beta is NULL");
    if (n_obs > 0 && (!obs || !obs_out)) return bad("obs and obs_out are needed for n_obs > 0");
    bool any = false;
    for (int b = 0; b < n_bins; ++b) {
        if (H[b] < 0) return bad("H[%d] is negative", b);
        if (H[b] > 0) {
            any = true;
            if (!std::isfinite(lnW[b])) return bad("lnW[%d] is not finite", b);
        }
    }
    if (!any) return bad("no visited bin (H is zero everywhere)");
    const double nan = std::numeric_limits<double>::quiet_NaN();
    for (int i = 0; i < n_beta; ++i) {
        const double bt = beta[i];
        if (!std::isfinite(bt)) return bad("beta[%d] is not finite", i);
        // ln of the unnormalised P_beta(E) per visited bin; shift by the maximum
        double mx = -INFINITY;
        for (int b = 0; b < n_bins; ++b)
            if (H[b] > 0) mx = std::max(mx, std::log((double)H[b]) - bt * (e_lo + b) - lnW[b]);
        double z = 0.0, m1 = 0.0, m2 = 0.0;
        for (int b = 0; b < n_bins; ++b) {
            if (H[b] <= 0) continue;
            const double e = (double)(e_lo + b);
            const double p = std::exp(std::log((double)H[b]) - bt * e - lnW[b] - mx);
            z += p;
            m1 += p * e;
            m2 += p * e * e;
        }
        if (mean_E) mean_E[i] = m1 / z;
        if (mean_E2) mean_E2[i] = m2 / z;
        for (int k = 0; k < n_obs; ++k) {
            const double *o = obs + (size_t)k * n_bins;
            double zk = 0.0, sk = 0.0;
            for (int b = 0; b < n_bins; ++b) {
                if (H[b] <= 0 || !std::isfinite(o[b])) continue;
                const double p = std::exp(std::log((double)H[b]) - bt * (e_lo + b) - lnW[b] - mx);
                zk += p;
                sk += p * o[b];
            }
            obs_out[(size_t)i * n_obs + k] = zk > 0.0 ? sk / zk : nan;
        }
    }
    return MUCAL_OK;
}

int mucal_multi_histogram(const int64_t *H, const double *lnW, int32_t K, int32_t n_bins,
                          int32_t max_iter, double tol, double *ln_omega, int32_t *iterations)
{
    if (!H || !lnW || !ln_omega) return bad("H, lnW and ln_omega must not be NULL");
    if (K < 1 || n_bins < 1) return bad("need K >= 1 and n_bins >= 1");
    if (max_iter < 1 || !(tol > 0.0)) return bad("need max_iter >= 1 and tol > 0");
    std::vector<double> lnN((size_t)K, -INFINITY), f((size_t)K, 0.0), fn((size_t)K, 0.0);
    std::vector<double> num((size_t)n_bins, 0.0);
    bool any = false;
    for (int k = 0; k < K; ++k) {
        double tot = 0.0;
        for (int b = 0; b < n_bins; ++b) {
            const int64_t h = H[(size_t)k * n_bins + b];
            if (h < 0) return bad("H[%d][%d] is negative", k, b);
            if (h > 0 && !std::isfinite(lnW[(size_t)k * n_bins + b]))
                return bad("lnW[%d][%d] is not finite", k, b);
            tot += (double)h;
            num[b] += (double)h;
        }
        if (tot > 0.0) lnN[k] = std::log(tot);
        any = any || tot > 0.0;
    }
    if (!any) return bad("every histogram is empty");
    const double nan = std::numeric_limits<double>::quiet_NaN();
    int it = 0;
    for (it = 1; it <= max_iter; ++it) {
        // ln Omega(E) = ln sum_k H_k(E) - ln sum_k N_k exp(lnW_k(E) - f_k)
        for (int b = 0; b < n_bins; ++b) {
            if (num[b] <= 0.0) {
                ln_omega[b] = nan;
                continue;
            }
            double mx = -INFINITY;
            for (int k = 0; k < K; ++k)
                if (std::isfinite(lnN[k])) mx = std::max(mx, lnN[k] + lnW[(size_t)k * n_bins + b] - f[k]);
            double sden = 0.0;
            for (int k = 0; k < K; ++k)
                if (std::isfinite(lnN[k])) sden += std::exp(lnN[k] + lnW[(size_t)k * n_bins + b] - f[k] - mx);
            ln_omega[b] = std::log(num[b]) - (mx + std::log(sden));
        }
        // f_k = ln sum_E Omega(E) exp(lnW_k(E)), shifted so that f_0 = 0
        for (int k = 0; k < K; ++k) {
            double mx = -INFINITY;
            for (int b = 0; b < n_bins; ++b)
                if (num[b] > 0.0) mx = std::max(mx, ln_omega[b] + lnW[(size_t)k * n_bins + b]);
            double sz = 0.0;
            for (int b = 0; b < n_bins; ++b)
                if (num[b] > 0.0) sz += std::exp(ln_omega[b] + lnW[(size_t)k * n_bins + b] - mx);
            fn[k] = mx + std::log(sz);
        }
        double delta = 0.0;
        const double f0 = fn[0];
        for (int k = 0; k < K; ++k) {
            fn[k] -= f0;
            delta = std::max(delta, std::fabs(fn[k] - f[k]));
            f[k] = fn[k];
        }
        if (delta < tol) break;
    }
    // shift ln Omega to maximum 0
    double mx = -INFINITY;
    for (int b = 0; b < n_bins; ++b)
        if (num[b] > 0.0) mx = std::max(mx, ln_omega[b]);
    for (int b = 0; b < n_bins; ++b)
        if (num[b] > 0.0) ln_omega[b] -= mx;
    if (iterations) *iterations = std::min(it, max_iter);
    return MUCAL_OK;
}

int mucal_ln_omega_normalise(double *ln_omega, int32_t n_bins, int64_t V, int64_t N)
{
    if (!ln_omega || n_bins < 1) return bad("need ln_omega and n_bins >= 1");
    if (V < 1 || N < 0 || N > V) return bad("need V >= 1 and 0 <= N <= V");
    // logsumexp over the finite entries, shifted by their maximum
    double mx = -INFINITY;
    for (int b = 0; b < n_bins; ++b)
        if (std::isfinite(ln_omega[b])) mx = std::max(mx, ln_omega[b]);
    if (!std::isfinite(mx)) return bad("no finite entry to normalise");
    double sum = 0.0;
    for (int b = 0; b < n_bins; ++b)
        if (std::isfinite(ln_omega[b])) sum += std::exp(ln_omega[b] - mx);
    const double lse = mx + std::log(sum);
    // ln C(V, N): every configuration has some energy
    const double ln_total = std::lgamma((double)V + 1.0) - std::lgamma((double)N + 1.0) -
                            std::lgamma((double)(V - N) + 1.0);
    for (int b = 0; b < n_bins; ++b)
        if (std::isfinite(ln_omega[b])) ln_omega[b] += ln_total - lse;
    return MUCAL_OK;
}

int mucal_ln_omega(const int64_t *H, const double *lnW, int32_t n_bins, int64_t V, int64_t N,
                   double *ln_omega)
{
    if (!H || !lnW || !ln_omega) return bad("H, lnW and ln_omega must not be NULL");
    if (n_bins < 1) return bad("n_bins must be >= 1");
    const double nan = std::numeric_limits<double>::quiet_NaN();
    bool any = false;
    for (int b = 0; b < n_bins; ++b) {
        if (H[b] < 0) return bad("H[%d] is negative", b);
        if (H[b] == 0) {
            ln_omega[b] = nan;
            continue;
        }
        if (!std::isfinite(lnW[b])) return bad("lnW[%d] is not finite", b);
        // W = 1/Omega makes H flat (Sec. 2): Omega(E) is proportional to H(E) / W(E)
        ln_omega[b] = std::log((double)H[b]) - lnW[b];
        any = true;
    }
    if (!any) return bad("no visited bin (H is zero everywhere)");
    return mucal_ln_omega_normalise(ln_omega, n_bins, V, N);
}

int mucal_ising_constant(int32_t d, int64_t V, int64_t N, double J, double *c_N)
{
    if (d != 2 && d != 3) return bad("d must be 2 or 3");
    if (V < 1 || N < 0 || N > V) return bad("need V >= 1 and 0 <= N <= V");
    if (!c_N) return bad("c_N is NULL");
    *c_N = J * (double)d * ((double)V / 4.0 - (double)N);
    return MUCAL_OK;
}

int mucal_droplet_delta(int32_t d, int64_t V, int64_t N, double rho0, double kappa_hat,
                        double tau_W, double *Delta, double *V_L)
{
    if (d != 2 && d != 3) return bad("d must be 2 or 3");
    if (V < 1 || N < 0) return bad("need V >= 1 and N >= 0");
    if (!(rho0 >= 0.0 && rho0 < 0.5)) return bad("rho0 must lie in [0, 1/2)");
    if (!(kappa_hat > 0.0) || !(tau_W > 0.0) || !std::isfinite(kappa_hat) || !std::isfinite(tau_W))
        return bad("kappa_hat and tau_W must be positive and finite");
    const double m0 = 1.0 - 2.0 * rho0;
    const double vl = ((double)N - rho0 * (double)V) / m0;                       // Eq. 8
    double delta = 0.0;
    if (vl > 0.0)
        delta = m0 * m0 / (2.0 * kappa_hat * tau_W) * std::pow(vl, (double)(d + 1) / d) / (double)V;  // Eq. 10
    if (Delta) *Delta = delta;
    if (V_L) *V_L = vl;
    return MUCAL_OK;
}

int mucal_droplet_lambda(int32_t d, double Delta, double *lambda)
{
    if (d != 2 && d != 3) return bad("d must be 2 or 3");
    if (!(Delta >= 0.0) || !std::isfinite(Delta)) return bad("Delta must be finite and >= 0");
    if (!lambda) return bad("lambda is NULL");
    *lambda = 0.0;
    if (Delta == 0.0) return MUCAL_OK;
    // Stationary points in (0, 1): lambda^(1/d) (1 - lambda) = (d-1) / (2 d Delta).
    // The left side rises up to lambda* = 1/(d+1) and falls to 0 at 1; the
    // local minimum of f is the root on the falling branch.
    const double rhs = (double)(d - 1) / (2.0 * d * Delta);
    const double inv_d = 1.0 / d;
    auto g = [&](double x) { return std::pow(x, inv_d) * (1.0 - x); };
    double lo = 1.0 / (d + 1), hi = 1.0;
    if (g(lo) < rhs) return MUCAL_OK;   // no interior stationary point: lambda = 0
    for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (g(mid) >= rhs)
            lo = mid;
        else
            hi = mid;
    }
    const double root = lo;
    if (droplet_free_energy(d, Delta, root) < droplet_free_energy(d, Delta, 0.0)) *lambda = root;
    return MUCAL_OK;
}

}  // extern "C"
