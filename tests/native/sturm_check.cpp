// Host build of the double-float Sturm count (csrc/sturm_df.h) used by the GPU
// bisection.  stdin: k, d[k], e[k-1], q, x[q]; stdout: the count below each x.
#include <cstdio>
#include <vector>

#include "sturm_df.h"

struct Pair {
    float x, y;
};

int main() {
    using namespace rsdft::dfl;
    int k = 0;
    if (std::scanf("%d", &k) != 1 || k < 1) return 1;
    std::vector<double> d(k), e(k > 1 ? k - 1 : 0);
    for (auto &v : d)
        if (std::scanf("%lf", &v) != 1) return 1;
    for (auto &v : e)
        if (std::scanf("%lf", &v) != 1) return 1;
    std::vector<Pair> dt(k), et(k);
    for (int i = 0; i < k; ++i) {
        const df a = from_double(d[i]);
        dt[i] = Pair{a.h, a.l};
    }
    for (int i = 0; i + 1 < k; ++i) {
        const df a = sqr(from_double(e[i]));
        et[i] = Pair{a.h, a.l};
    }
    int q = 0;
    if (std::scanf("%d", &q) != 1) return 1;
    for (int j = 0; j < q; ++j) {
        double x = 0.0;
        if (std::scanf("%lf", &x) != 1) return 1;
        std::printf("%d\n", sturm_count_df(dt.data(), et.data(), k, from_double(x)));
    }
    return 0;
}
