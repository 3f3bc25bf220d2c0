// Sturm count of a real symmetric tridiagonal T in double-float (dfloat.h): the
// number of eigenvalues of T below x, as the number of sign changes of the
// leading principal minors p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2} (p_{-1} = 1).
// An exact p_i = 0 counts as negative (replaced by -p_{i-1} 2^-50); p_i and p_{i-1}
// are scaled by one power of two whenever the larger leaves [2^-60, 2^60] (exact;
// FP32's exponent range is much narrower than FP64's).  dt[i] = d_i and
// et[i] = e_i^2 as (hi, lo) pairs in any type with members x and y.  Host and
// device (the host build is the CPU check of the device code).
#pragma once
#include "dfloat.h"

namespace rsdft {
namespace dfl {

template <typename F2>
DF_FN int sturm_count_df(const F2 *dt, const F2 *et, int k, df x) {
    df pm{1.0f, 0.0f};
    df p = sub(df{dt[0].x, dt[0].y}, x);
    if (p.h == 0.0f) p = df{-0x1p-50f, 0.0f};
    int cnt = p.h < 0.0f ? 1 : 0;
    for (int i = 1; i < k; ++i) {
        const df t = sub(df{dt[i].x, dt[i].y}, x);
        df pn = sub(mul(t, p), mul(df{et[i - 1].x, et[i - 1].y}, pm));
        if (pn.h == 0.0f) pn = mul_f(neg(p), 0x1p-50f);
        cnt += (pn.h < 0.0f) != (p.h < 0.0f) ? 1 : 0;
        const int ea = fexp(pn.h), eb = fexp(p.h);
        const int ex = ea > eb ? ea : eb;
        if (ex > 60 || ex < -60) {
            const float sc = ffrombits((127 - ex) << 23);   // 2^-ex
            pn = mul_f(pn, sc);
            p = mul_f(p, sc);
        }
        pm = p;
        p = pn;
    }
    return cnt;
}

}  // namespace dfl
}  // namespace rsdft
