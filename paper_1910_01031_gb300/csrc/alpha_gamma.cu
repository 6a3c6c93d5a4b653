// The one-stage IEWPF's alpha from the incomplete-gamma form of the implicit
// equation (App. A, eq. numericalEqForAlpha):
//     P(N_psi/2, alpha gamma/2) = exp(-c*/2) P(N_psi/2, gamma/2),
// P the regularised lower incomplete gamma function (the ratio of two lower
// incomplete gamma functions equals the ratio of their regularised forms).
// Everything is carried in logarithms, so the gamma functions cannot
// overflow for large N_psi; the cost grows like sqrt(N_psi) per evaluation.
#include <math.h>

#include "kernels.h"

namespace iewpf {
namespace {

constexpr int GAMMA_MAX_TERMS = 400000;

// log P(s, x) for s > 0, x > 0.  x < s + 1: the power series
//     P(s, x) = x^s e^{-x} / Gamma(s + 1) * sum_{n>=0} x^n / ((s+1)...(s+n))
// (Abramowitz & Stegun 6.5.4 with 6.5.29).  Otherwise Q = 1 - P from the
// continued fraction of the upper function (A&S 6.5.31),
//     Q(s, x) = x^s e^{-x} / Gamma(s) / (x + 1 - s - 1(1 - s)/(x + 3 - s - 2(2 - s)/(x + 5 - s - ...))),
// evaluated by the modified Lentz method (Thompson & Barnett 1986), and
// log P = log1p(-Q).  *ok is cleared when the series or fraction does not
// settle within GAMMA_MAX_TERMS.
__device__ double log_gamma_p(double s, double x, bool* ok)
{
    const double pre = s * log(x) - x;
    if (x < s + 1.0) {
        double term = 1.0, sum = 1.0;
        int n = 1;
        for (; n < GAMMA_MAX_TERMS; ++n) {
            term *= x / (s + n);
            sum += term;
            if (term < sum * 1e-17) break;
        }
        if (n >= GAMMA_MAX_TERMS) *ok = false;
        return pre - lgamma(s + 1.0) + log(sum);
    }
    const double tiny = 1e-300;
    double b = x + 1.0 - s, c = 1.0 / tiny, d = 1.0 / b, h = d;
    int i = 1;
    for (; i < GAMMA_MAX_TERMS; ++i) {
        const double an = -i * (i - s);
        b += 2.0;
        d = an * d + b;
        if (fabs(d) < tiny) d = tiny;
        c = b + an / c;
        if (fabs(c) < tiny) c = tiny;
        d = 1.0 / d;
        const double del = d * c;
        h *= del;
        if (fabs(del - 1.0) < 1e-16) break;
    }
    if (i >= GAMMA_MAX_TERMS) *ok = false;
    return log1p(-exp(pre - lgamma(s) + log(h)));
}

// alpha_i: y = alpha gamma/2 solves log P(s, y) = log P(s, gamma/2) - c*/2,
// s = N_psi/2, on (0, gamma/2] (log P increases with y): a bracket from
// halving, then Newton steps kept inside it (bisection when a step leaves).
__global__ void alpha_gamma_kernel(int ne, double N, const double* __restrict__ gamma,
                                   const double* __restrict__ cstar, double* __restrict__ alpha, int* flag)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    const double s = 0.5 * N, g = gamma[i], cs = cstar[i];
    if (!(g > 0.0) || !(cs >= 0.0) || !isfinite(g) || !isfinite(cs)) {
        alpha[i] = nan("");
        atomicOr(flag, FLAG_DOMAIN);
        return;
    }
    if (cs == 0.0) {
        alpha[i] = 1.0;
        return;
    }
    bool ok = true;
    double hi = 0.5 * g;
    const double target = log_gamma_p(s, hi, &ok) - 0.5 * cs;
    double lo = 0.5 * hi;
    int k = 0;
    for (; k < 2100 && log_gamma_p(s, lo, &ok) >= target; ++k) {
        hi = lo;
        lo *= 0.5;
    }
    if (k >= 2100) ok = false;
    double y = 0.5 * (lo + hi);
    const double lgs = lgamma(s);
    for (int it = 0; it < 200 && ok; ++it) {
        const double lp = log_gamma_p(s, y, &ok);
        const double f = lp - target;
        if (f < 0.0) lo = y;
        else hi = y;
        // d/dy log P(s, y) = y^{s-1} e^{-y} / (Gamma(s) P(s, y))
        const double fp = exp((s - 1.0) * log(y) - y - lgs - lp);
        double yn = y - f / fp;
        if (!(yn > lo && yn < hi)) yn = 0.5 * (lo + hi);
        if (fabs(yn - y) <= 1e-15 * y || hi - lo <= 1e-15 * hi) {
            y = yn;
            break;
        }
        y = yn;
    }
    const double a = 2.0 * y / g;
    alpha[i] = a;
    if (!ok || !(a > 0.0) || !(a <= 1.0)) atomicOr(flag, FLAG_DOMAIN);
}

}  // namespace

cudaError_t launch_alpha_gamma(int ne, double N_psi, const double* gamma, const double* cstar, double* alpha,
                               int* flag, cudaStream_t st)
{
    if (ne <= 0) return cudaSuccess;
    alpha_gamma_kernel<<<(ne + 63) / 64, 64, 0, st>>>(ne, N_psi, gamma, cstar, alpha, flag);
    return cudaGetLastError();
}

}  // namespace iewpf
