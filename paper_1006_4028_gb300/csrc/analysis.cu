// Host-side analysis of solved correlators: effective masses and fits of
// one- or two-sided exponentials.  The paper plots effective masses of C_PP
// (Sec. III, the heavy-quark demonstration) without writing a definition
// out; the two readings here are the log ratio and the cosh form for a state
// that propagates both ways round the periodic time direction.
//
// No GPU work: T values in, a few values out, plain double arithmetic with
// fixed iteration counts (bisection, a log-spaced scan and golden-section
// search), so the results are reproducible bit for bit on any host.
#include <cmath>

#include "ctx.h"
#include "dpre.h"

namespace {

double log_cosh(double x)
{
    x = std::fabs(x);
    return x + std::log1p(std::exp(-2.0 * x)) - std::log(2.0);
}

// m > 0 with log cosh(m a) - log cosh(m b) = log r; NaN if none in (0, 50]
double cosh_mass(double r, double a, double b)
{
    if (!(r > 0) || !std::isfinite(r)) return NAN;
    const double lr = std::log(r);
    auto f = [&](double m) { return log_cosh(m * a) - log_cosh(m * b) - lr; };
    double lo = 1e-12, hi = 50.0;
    double flo = f(lo), fhi = f(hi);
    if (!(flo * fhi < 0)) return NAN;
    for (int it = 0; it < 200 && hi - lo > 1e-16 * hi; it++) {
        const double mid = 0.5 * (lo + hi);
        const double fm = f(mid);
        if ((fm < 0) == (flo < 0)) {
            lo = mid;
            flo = fm;
        } else {
            hi = mid;
        }
    }
    return 0.5 * (lo + hi);
}

// model shape f(m, t) without the amplitude
double shape(int kind, double m, int t, int T)
{
    double v = std::exp(-m * t);
    if (kind == 1) v += std::exp(-m * (T - t));
    return v;
}

// sum over the window of (A f/C - 1)^2 with A at its closed-form minimum
// A = sum(g) / sum(g^2), g = f/C
double fit_cost(const double *c, int T, int kind, int t0, int t1, double m, double *A_out)
{
    double sg = 0, sg2 = 0;
    for (int t = t0; t <= t1; t++) {
        const double g = shape(kind, m, t, T) / c[t];
        sg += g;
        sg2 += g * g;
    }
    const double A = sg2 > 0 ? sg / sg2 : 0.0;
    double r = 0;
    for (int t = t0; t <= t1; t++) {
        const double d = A * shape(kind, m, t, T) / c[t] - 1.0;
        r += d * d;
    }
    if (A_out) *A_out = A;
    return r;
}

}  // namespace

extern "C" {

dp_status dp_effective_mass(const double *c, int T, int kind, double *m_out)
{
    if (!c || !m_out || T < 2 || (kind != 0 && kind != 1)) {
        dp::set_error("effective mass needs c[T], m_out[T-1], T >= 2 and kind 0 or 1");
        return DP_ERR_INVALID_ARG;
    }
    for (int t = 0; t + 1 < T; t++) {
        const double r = c[t] / c[t + 1];
        if (kind == 0)
            m_out[t] = (r > 0 && std::isfinite(r)) ? std::log(r) : NAN;
        else
            m_out[t] = cosh_mass(r, 0.5 * T - t, 0.5 * T - t - 1.0);
    }
    return DP_OK;
}

dp_status dp_pcac_mass(const double *cpp, const double *cap, int T, double *m_out)
{
    if (!cpp || !cap || !m_out || T < 3) {
        dp::set_error("PCAC mass needs cpp[T], cap[T], m_out[T] and T >= 3");
        return DP_ERR_INVALID_ARG;
    }
    m_out[0] = m_out[T - 1] = NAN;
    for (int t = 1; t + 1 < T; t++)
        m_out[t] = (cap[t + 1] - cap[t - 1]) / (4.0 * cpp[t]);
    return DP_OK;
}

dp_status dp_fit_correlator(const double *c, int T, int kind, int t0, int t1, double *m_out,
                            double *A_out, double *rms_out)
{
    if (!c || !m_out || (kind != 0 && kind != 1) || t0 < 0 || t1 >= T || t1 - t0 < 1) {
        dp::set_error("fit needs c[T], 0 <= t0 < t1 < T and kind 0 or 1");
        return DP_ERR_INVALID_ARG;
    }
    for (int t = t0; t <= t1; t++)
        if (!std::isfinite(c[t]) || c[t] == 0.0 || (c[t] > 0) != (c[t0] > 0)) {
            dp::set_error("fit window holds a zero, a non-finite value or a sign change");
            return DP_ERR_INVALID_ARG;
        }
    // coarse scan on a log grid over [1e-4, 20], then golden-section search
    // between the best point's neighbours
    const int N = 400;
    const double lmin = std::log(1e-4), lmax = std::log(20.0);
    int best = 0;
    double bcost = INFINITY;
    for (int i = 0; i <= N; i++) {
        const double m = std::exp(lmin + (lmax - lmin) * i / N);
        const double r = fit_cost(c, T, kind, t0, t1, m, nullptr);
        if (r < bcost) {
            bcost = r;
            best = i;
        }
    }
    double lo = std::exp(lmin + (lmax - lmin) * (best > 0 ? best - 1 : 0) / N);
    double hi = std::exp(lmin + (lmax - lmin) * (best < N ? best + 1 : N) / N);
    const double gr = 0.5 * (std::sqrt(5.0) - 1.0);
    double x1 = hi - gr * (hi - lo), x2 = lo + gr * (hi - lo);
    double f1 = fit_cost(c, T, kind, t0, t1, x1, nullptr), f2 = fit_cost(c, T, kind, t0, t1, x2, nullptr);
    for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; it++) {
        if (f1 <= f2) {
            hi = x2;
            x2 = x1;
            f2 = f1;
            x1 = hi - gr * (hi - lo);
            f1 = fit_cost(c, T, kind, t0, t1, x1, nullptr);
        } else {
            lo = x1;
            x1 = x2;
            f1 = f2;
            x2 = lo + gr * (hi - lo);
            f2 = fit_cost(c, T, kind, t0, t1, x2, nullptr);
        }
    }
    const double m = 0.5 * (lo + hi);
    double A = 0;
    const double cost = fit_cost(c, T, kind, t0, t1, m, &A);
    *m_out = m;
    if (A_out) *A_out = A;
    if (rms_out) *rms_out = std::sqrt(cost / (t1 - t0 + 1));
    return DP_OK;
}

}  // extern "C"
