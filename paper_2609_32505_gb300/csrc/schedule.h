// Polynomial schedules for the polar iteration X <- X (c1 I + c3 X^T X).
//
// The degree-3 CANS step on an interval [a, b] (Appendix A.4 / B.8) is the odd
// cubic p(x) = c1 x + c3 x^3 with the smallest max_{[a,b]} |1 - p(x)|.  By
// Chebyshev equioscillation the error alternates at a, at the interior maximum
// e (p'(e) = 0) and at b, which gives in closed form
//   s = a^2 + ab + b^2,  e = sqrt(s/3),  c3 = -c1/s,
//   c1 = 2 / ((2/3) e + ab(a+b)/s),  E = (2/3) c1 e - 1,
// and p maps [a, b] onto [1 - E, 1 + E].  Preprocessing (Appendix B.8) finds the
// largest [t, 1] that `pre` such greedy steps map into [1 - delta, 1 + delta];
// the main iteration then starts from [1 - delta, 1 + delta].
#pragma once
#include <cmath>
#include <vector>

namespace psvd {

struct Cubic { double c1, c3, e; };

__host__ __device__ inline Cubic cans_cubic(double a, double b) {
    const double s = a * a + a * b + b * b;
    const double e = sqrt(s / 3.0);
    const double c1 = 2.0 / ((2.0 / 3.0) * e + a * b * (a + b) / s);
    return Cubic{c1, -c1 / s, (2.0 / 3.0) * c1 * e - 1.0};
}

// Interval half-width after `steps` greedy cubics starting from [a, 1].
__host__ __device__ inline double greedy_width(double a, int steps) {
    double lo = a, hi = 1.0, e = 1.0 - a;
    for (int i = 0; i < steps; ++i) {
        Cubic c = cans_cubic(lo, hi);
        e = c.e;
        lo = 1.0 - e;
        hi = 1.0 + e;
    }
    return e;
}

// Conservative CANS schedule: `pre` preprocessing cubics for [t, 1], then greedy
// cubics from [1 - delta, 1 + delta]; `total` coefficient pairs in all.
// Returns t through *t_out.
inline std::vector<Cubic> cans_schedule(double delta, int pre, int total, double *t_out = nullptr) {
    std::vector<Cubic> out;
    double t = 1.0 - delta;
    if (pre > 0) {
        // bisection on log t: the width after `pre` steps decreases as t grows
        double lo = 1e-300, hi = 1.0;
        for (int it = 0; it < 200; ++it) {
            const double mid = std::sqrt(lo * hi);
            if (greedy_width(mid, pre) <= delta) hi = mid; else lo = mid;
        }
        t = hi;
        double a = t, b = 1.0;
        for (int i = 0; i < pre && (int)out.size() < total; ++i) {
            Cubic c = cans_cubic(a, b);
            out.push_back(c);
            a = 1.0 - c.e;
            b = 1.0 + c.e;
        }
    }
    double a = 1.0 - delta, b = 1.0 + delta;
    while ((int)out.size() < total) {
        Cubic c = cans_cubic(a, b);
        out.push_back(c);
        a = 1.0 - c.e;
        b = 1.0 + c.e;
    }
    if (t_out) *t_out = t;
    return out;
}

// Damped greedy cubic (the Polar-Express-style comparison schedule of the polar-iteration
// ablation, Appendix B): the optimal cubic p for [a, b] applied to x / damp, i.e.
// coefficients (c1 / damp, c3 / damp^3); the image of [a, b] under x -> p(x / damp) is
// returned in [*lo, *hi] (p rises up to its interior maximum e and falls after it).
__host__ __device__ inline Cubic damped_cubic(double a, double b, double damp, double *lo, double *hi) {
    const Cubic c = cans_cubic(a, b);
    auto p = [&](double y) { return c.c1 * y + c.c3 * y * y * y; };
    const double ya = a / damp, yb = b / damp, e = sqrt(-c.c1 / (3.0 * c.c3));
    double mn = fmin(p(ya), p(yb)), mx = fmax(p(ya), p(yb));
    if (e > ya && e < yb) mx = fmax(mx, p(e));
    *lo = mn;
    *hi = mx;
    return Cubic{c.c1 / damp, c.c3 / (damp * damp * damp), c.e};
}

// Steps of a greedy schedule from [a, 1] until the interval half-width is <= w.
__host__ __device__ inline int greedy_steps_to(double a, double w, int cap) {
    double lo = a, hi = 1.0;
    for (int k = 0; k < cap; ++k) {
        if (hi - 1.0 <= w && 1.0 - lo <= w) return k;
        Cubic c = cans_cubic(lo, hi);
        lo = 1.0 - c.e;
        hi = 1.0 + c.e;
    }
    return cap;
}

}  // namespace psvd
