// Host-side numerics of the library: Chebyshev filter construction (Sec. 2.2.1, Eqs. (2.4)-
// (2.7)), the KPM density and DOS slicer (Sec. 2.1, Eq. (2.2)), and the inertia count of the
// arrowhead-plus-tridiagonal projected matrix used by the bisection eigensolver.
#include <algorithm>
#include <cmath>
#include <vector>

#include "evsl_internal.h"

namespace {

enum class Kind { Interior, Left, Right };

// Damping multipliers g_0..g_k for a degree-k expansion (Eq. (2.6) for Lanczos sigma;
// Jackson: g_j = ((k - j + 2) cos(j a) + sin(j a) cot(a)) / (k + 2), a = pi / (k + 2)).
void damping_factors(evsl_damping kind, int k, std::vector<double> &g)
{
    g.assign(k + 1, 1.0);
    if (kind == EVSL_DAMP_SIGMA) {
        const double th = M_PI / (k + 1);
        for (int j = 1; j <= k; ++j) g[j] = std::sin(j * th) / (j * th);
    } else if (kind == EVSL_DAMP_JACKSON) {
        const double a = M_PI / (k + 2);
        const double cot = std::cos(a) / std::sin(a);
        for (int j = 1; j <= k; ++j) g[j] = ((k - j + 2) * std::cos(j * a) + std::sin(j * a) * cot) / (k + 2);
    }
}

// T_j(t) for j = 0..k from the definition (trigonometric inside [-1, 1], hyperbolic outside)
void cheb_values(double t, int k, std::vector<double> &out)
{
    out.resize(k + 1);
    if (std::fabs(t) <= 1.0) {
        const double th = std::acos(t);
        for (int j = 0; j <= k; ++j) out[j] = std::cos(j * th);
    } else {
        const double ph = std::acosh(std::fabs(t));
        const double sg = t < 0 ? -1.0 : 1.0;
        for (int j = 0; j <= k; ++j) out[j] = ((j & 1) ? sg : 1.0) * std::cosh(j * ph);
    }
}

struct Filter {
    int k;
    std::vector<double> g, Ta, Tb;
    // P(t) for the expansion centred at angle th: sum_j g_j m_j T_j(t), m_0 = 1/2, m_j = cos(j th)
    double eval(const std::vector<double> &T, double th) const
    {
        double s = 0.5 * g[0] * T[0];
        for (int j = 1; j <= k; ++j) s += g[j] * std::cos(j * th) * T[j];
        return s;
    }
    double at_centre(double th) const
    {
        double s = 0.5 * g[0];
        for (int j = 1; j <= k; ++j) {
            const double cj = std::cos(j * th);
            s += g[j] * cj * cj;  // T_j(cos th) = cos(j th)
        }
        return s;
    }
    // balance function f(th) = P(ta) - P(tb) (the j = 0 terms cancel) and its derivative
    void balance(double th, double *f, double *df) const
    {
        double s = 0.0, ds = 0.0;
        for (int j = 1; j <= k; ++j) {
            const double diff = Ta[j] - Tb[j];
            s += g[j] * std::cos(j * th) * diff;
            ds -= g[j] * j * std::sin(j * th) * diff;
        }
        *f = s;
        *df = ds;
    }
};

// Newton's method on th in [acos(tb), acos(ta)], kept inside a shrinking sign-change bracket.
double balanced_angle(const Filter &F, double ta, double tb)
{
    double left = std::acos(tb), right = std::acos(ta);
    double fl, fr, d;
    F.balance(left, &fl, &d);
    F.balance(right, &fr, &d);
    double th = 0.5 * (left + right);
    if ((fl > 0) == (fr > 0)) return th;  // no sign change: use the interval centre
    const bool left_negative = fl < 0;
    for (int it = 0; it < 200; ++it) {
        double f, df;
        F.balance(th, &f, &df);
        if ((f < 0) == left_negative)
            left = th;
        else
            right = th;
        double next = (df != 0.0) ? th - f / df : 0.5 * (left + right);
        if (!(next > left && next < right)) next = 0.5 * (left + right);
        const double moved = std::fabs(next - th);
        th = next;
        if (moved < 1e-14) break;
    }
    return th;
}

}  // namespace

int host_filter_build(double a, double b, double lmin, double lmax, const evsl_filter_opts *o,
                      evsl_polfilt *pol, double *coef, int cap)
{
    evsl_filter_opts opt = {0.8, 0.4, EVSL_DAMP_JACKSON, 10000};
    if (o) opt = *o;
    if (!pol || !(b > a) || !(lmax > lmin) || opt.max_deg < 2 || !(opt.tau > 0) ||
        !(opt.tau_ext > 0))
        return EVSL_ERR_ARG;
    const double c = 0.5 * (lmax + lmin), d = 0.5 * (lmax - lmin);
    const double ta = (a - c) / d, tb = (b - c) / d;
    Kind kind = Kind::Interior;
    if (ta <= -1.0 && tb >= 1.0) return EVSL_ERR_ARG;  // covers the whole spectrum
    if (tb <= -1.0 || ta >= 1.0) return EVSL_ERR_ARG;  // outside the spectral interval
    if (ta <= -1.0) kind = Kind::Left;
    else if (tb >= 1.0) kind = Kind::Right;

    Filter F;
    double th = 0.0, bar = 0.0, norm = 1.0;
    int status = EVSL_ERR_NOCONV;
    for (int k = 2; k <= opt.max_deg; ++k) {
        F.k = k;
        damping_factors(opt.damping, k, F.g);
        if (kind == Kind::Interior) {
            cheb_values(ta, k, F.Ta);
            cheb_values(tb, k, F.Tb);
            th = balanced_angle(F, ta, tb);
            norm = F.at_centre(th);
            bar = F.eval(F.Ta, th) / norm;
            if (bar <= opt.tau) { status = EVSL_OK; break; }
        } else {
            th = (kind == Kind::Left) ? M_PI : 0.0;
            cheb_values(kind == Kind::Left ? tb : ta, k, F.Tb);
            norm = F.at_centre(th);
            bar = F.eval(F.Tb, th) / norm;
            if (bar <= opt.tau_ext) { status = EVSL_OK; break; }
        }
    }
    const int k = F.k;
    pol->deg = k;
    pol->boundary = (kind == Kind::Left) ? -1 : (kind == Kind::Right ? 1 : 0);
    pol->gamma = std::cos(th);
    pol->bar = bar;
    pol->lmin = lmin;
    pol->lmax = lmax;
    pol->a = a;
    pol->b = b;
    pol->coef = coef;
    if (!coef || cap < k + 1) return EVSL_ERR_CAPACITY;
    coef[0] = 0.5 * F.g[0] / norm;
    for (int j = 1; j <= k; ++j) coef[j] = F.g[j] * std::cos(j * th) / norm;
    return status;
}

namespace {

// Jackson-damped cumulative count on [lmin, t]:
// N(t) = (1/pi) [ g_0 mu_0 (pi - th) - 2 sum_{k>=1} g_k mu_k sin(k th) / k ],
// th = arccos of the mapped point (clamped to [-1, 1]), g the Jackson factors of degree M.
struct Dos {
    int M;
    double c, d;
    std::vector<double> gmu;
    Dos(const double *mu, int M_, double lmin, double lmax) : M(M_)
    {
        c = 0.5 * (lmax + lmin);
        d = 0.5 * (lmax - lmin);
        std::vector<double> g;
        damping_factors(EVSL_DAMP_JACKSON, M, g);
        gmu.resize(M + 1);
        for (int k = 0; k <= M; ++k) gmu[k] = g[k] * mu[k];
    }
    double count(double t) const
    {
        double x = (t - c) / d;
        x = std::min(1.0, std::max(-1.0, x));
        const double th = std::acos(x);
        double s = gmu[0] * (M_PI - th);
        for (int k = 1; k <= M; ++k) s -= 2.0 * gmu[k] * std::sin(k * th) / k;
        return s / M_PI;
    }
};

}  // namespace

int host_slicer(const double *mu, int degree, int64_t n, double lmin, double lmax, double xi,
                double eta, int ns, int npts, double *sli, double *est)
{
    (void)n;
    if (!mu || !sli || !est || degree < 0 || ns < 1 || !(eta > xi) || !(lmax > lmin))
        return EVSL_ERR_ARG;
    if (npts <= 0) npts = std::max(2001, 100 * ns);
    if (npts < 2) return EVSL_ERR_ARG;
    Dos dos(mu, degree, lmin, lmax);
    std::vector<double> xs(npts), cum(npts);
    for (int j = 0; j < npts; ++j) {
        xs[j] = xi + (eta - xi) * j / (npts - 1);
        cum[j] = dos.count(xs[j]) ;
    }
    const double base = cum[0], total = cum[npts - 1] - base;
    sli[0] = xi;
    sli[ns] = eta;
    int j = 1;
    for (int i = 1; i < ns; ++i) {
        const double want = total * i / ns;
        while (j < npts - 1 && cum[j] - base < want) ++j;
        const double lo = cum[j - 1] - base, hi = cum[j] - base;
        double frac = hi > lo ? (want - lo) / (hi - lo) : 1.0;
        frac = std::min(1.0, std::max(0.0, frac));
        sli[i] = xs[j - 1] + frac * (xs[j] - xs[j - 1]);
    }
    for (int i = 0; i < ns; ++i) est[i] = dos.count(sli[i + 1]) - dos.count(sli[i]);
    return EVSL_OK;
}

int host_count_below(int k, int l, const double *d, const double *e, double sigma)
{
    double emax = 1.0;
    for (int i = 0; i < k; ++i) emax = std::max(emax, e[i] * e[i]);
    const double pmin = 1e-290 * emax;
    int neg = 0;
    double schur = 0.0;
    for (int i = 0; i < l; ++i) {
        double p = d[i] - sigma;
        if (std::fabs(p) < pmin) p = -pmin;
        neg += p < 0.0;
        schur += e[i] * e[i] / p;
    }
    if (l >= k) return neg;
    double pm = 1.0, p = d[l] - sigma - schur;
    if (std::fabs(p) < pmin) p = -pmin;
    neg += p < 0.0;
    for (int i = l + 1; i < k; ++i) {
        double pn = (d[i] - sigma) * p - e[i - 1] * e[i - 1] * pm;
        if (pn == 0.0) pn = -pmin * p;  // a zero pivot counts as negative
        neg += (pn < 0.0) != (p < 0.0);
        pm = p;
        p = pn;
        const double ap = std::fabs(p);
        if (ap > 0x1p+600) {
            p *= 0x1p-600;
            pm *= 0x1p-600;
        } else if (ap < 0x1p-600) {
            p *= 0x1p+600;
            pm *= 0x1p+600;
        }
    }
    return neg;
}

// ------------------------------------------------------------------------------------------
// Slices with equal counts under the Lanczos quadrature density.  The cumulative count
// N(t) = (n / nvec) sum of the weights of the nodes <= t is a step function; with C0 = N just
// below xi and C1 = N(eta), boundary t_i (0 < i < ns) lies midway between the first node in
// [xi, eta] at which N reaches C0 + (i / ns)(C1 - C0) and the node before it (xi if none).
int host_slicer_landos(const double *nodes, const double *weights, const int *mused, int m, int nvec,
                       int64_t n, double xi, double eta, int ns, double *sli, double *est)
{
    std::vector<std::pair<double, double>> nw;
    for (int l = 0; l < nvec; l++)
        for (int j = 0; j < mused[l]; j++)
            nw.emplace_back(nodes[(size_t)l * m + j], weights[(size_t)l * m + j] * (double)n / (double)nvec);
    std::stable_sort(nw.begin(), nw.end(), [](const std::pair<double, double> &x, const std::pair<double, double> &y) {
        return x.first < y.first;
    });
    double c0 = 0.0, c1 = 0.0;
    int first = -1, last = -1;
    for (int i = 0; i < (int)nw.size(); i++) {
        if (nw[i].first < xi) c0 += nw[i].second;
        if (nw[i].first <= eta) c1 += nw[i].second;
        if (nw[i].first >= xi && nw[i].first <= eta) {
            if (first < 0) first = i;
            last = i;
        }
    }
    if (first < 0) return EVSL_ERR_ARG;
    sli[0] = xi;
    sli[ns] = eta;
    double cum = c0;
    int p = first;
    for (int s = 1; s < ns; s++) {
        const double target = c0 + (double)s / ns * (c1 - c0);
        while (p <= last && cum + nw[p].second < target) cum += nw[p++].second;
        if (p > last) p = last;
        const double prev = (p > first) ? nw[p - 1].first : xi;
        sli[s] = 0.5 * (prev + nw[p].first);
    }
    for (int s = 0; s < ns; s++) {
        double lo = 0.0, hi = 0.0;
        for (const auto &q : nw) {
            if (q.first < sli[s]) lo += q.second;
            if (s + 1 == ns ? q.first <= sli[s + 1] : q.first < sli[s + 1]) hi += q.second;
        }
        est[s] = hi - lo;
    }
    return EVSL_OK;
}
