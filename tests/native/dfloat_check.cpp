// Host check of the double-float building blocks (csrc/dfloat.h) against long
// double.  Prints, per operation, the largest error over random operands in
// units of u^2 = 2^-48 of the bound's scale: |x| + |y| for the sum (which may
// cancel), the exact result for the others; and the largest |lo| / ulp(hi) of
// a sum (renormalisation).
#include <cmath>
#include <cstdint>
#include <cstdio>

#include "dfloat.h"

using namespace rsdft::dfl;

static uint64_t state = 0x243F6A8885A308D3ull;
static double urand() {   // splitmix64 -> [0, 1)
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1p-53;
}
static df rand_df(int emin, int emax) {
    const double m = 1.0 + urand();
    const int e = emin + (int)(urand() * (emax - emin + 1));
    return from_double(std::ldexp(m, e) * (urand() < 0.5 ? -1.0 : 1.0));
}
static long double val(df x) { return (long double)x.h + (long double)x.l; }

int main() {
    const long double u2 = 0x1p-48L;
    long double w_add = 0, w_norm = 0, w_mul = 0, w_div = 0, w_sqrt = 0, w_sqr = 0, w_cmul = 0;
    for (int t = 0; t < 200000; ++t) {
        const df x = rand_df(-20, 20);
        // y close to -x in a quarter of the cases (cancellation)
        df y = rand_df(-20, 20);
        if (t % 4 == 0) y = neg(mul(x, from_double(1.0 + std::ldexp(urand() - 0.5, -(int)(urand() * 40)))));
        const long double X = val(x), Y = val(y);
        const df s = add(x, y);
        w_add = std::fmax(w_add, std::fabs(val(s) - (X + Y)) / ((std::fabs(X) + std::fabs(Y)) * u2));
        if (s.h != 0.0f)
            w_norm = std::fmax(w_norm, std::fabs((long double)s.l) / (std::fabs((long double)s.h) * 0x1p-24L));
        const df p = mul(x, y);
        w_mul = std::fmax(w_mul, std::fabs(val(p) - X * Y) / (std::fabs(X * Y) * u2));
        const df q = div(x, y);
        w_div = std::fmax(w_div, std::fabs(val(q) - X / Y) / (std::fabs(X / Y) * u2));
        const df ax = x.h < 0.0f ? neg(x) : x;
        const long double R = sqrtl(val(ax));
        w_sqrt = std::fmax(w_sqrt, std::fabs(val(rsdft::dfl::sqrt(ax)) - R) / (R * u2));
        w_sqr = std::fmax(w_sqr, std::fabs(val(sqr(x)) - X * X) / (X * X * u2));
        // complex product, error relative to |a| |b|
        const cdf a{x, y}, b{rand_df(-5, 5), rand_df(-5, 5)};
        const cdf c = cmul(a, b);
        const long double ar = val(a.re), ai = val(a.im), br = val(b.re), bi = val(b.im);
        const long double cr = ar * br - ai * bi, ci = ar * bi + ai * br;
        const long double scale = sqrtl((ar * ar + ai * ai) * (br * br + bi * bi));
        w_cmul = std::fmax(w_cmul, std::fmax(std::fabs(val(c.re) - cr), std::fabs(val(c.im) - ci)) / (scale * u2));
    }
    std::printf("add %.3Lf\nnorm %.3Lf\nmul %.3Lf\ndiv %.3Lf\nsqrt %.3Lf\nsqr %.3Lf\ncmul %.3Lf\n", w_add, w_norm,
                w_mul, w_div, w_sqrt, w_sqr, w_cmul);
    return 0;
}
