// taps.cu -- the fetch tables of in-ray tap smoothing (Section 4.2, Algorithm 9), on the
// host: the binomial filters b_n and the linear-sampling fold that turns a symmetric
// discrete kernel into the (c0, offsets, weights) of SHW_SMOOTH_TAPS.
//
// Linear sampling: two neighbouring taps a and a+1 of weights w_a, w_{a+1} equal one
// linearly interpolated fetch of weight w_a + w_{a+1} at the point a + w_{a+1}/(w_a +
// w_{a+1}) between them, because interpolation at that point mixes the two values in the
// ratio of their weights.  An N-tap kernel (radius r = (N-1)/2) therefore needs 1 + 2 ceil(r/2)
// fetches per axis instead of N; Algorithm 9 prints the result for a 9-tap kernel.
#include <cmath>
#include <cstdint>

#include "shw.h"

namespace {

// Pascal's row n (n <= 62: every entry and the row sum 2^n fit in 64 bits).
void pascal_row(int n, uint64_t *row)
{
    row[0] = 1;
    for (int i = 1; i <= n; ++i) {
        row[i] = 1;
        for (int k = i - 1; k > 0; --k) row[k] += row[k - 1];
    }
}

}  // namespace

extern "C" {

shw_status shw_linear_sampling_taps(const double *w_host, int32_t radius, double *c0, double *offsets,
                                    double *weights, int32_t capacity, int32_t *nfetch)
{
    if (!w_host || !c0 || !offsets || !weights || !nfetch || radius < 0 || radius > 64) return SHW_EINVAL;
    const int need = (radius + 1) / 2;
    if (capacity < need) return SHW_ENOMEM;
    for (int k = 0; k <= 2 * radius; ++k)
        if (!std::isfinite(w_host[k])) return SHW_EINVAL;
    for (int k = 1; k <= radius; ++k)
        if (w_host[radius + k] != w_host[radius - k]) return SHW_EINVAL;  // the kernel must be symmetric
    int j = 0;
    for (int a = 1; a <= radius; a += 2, ++j) {
        const double wa = w_host[radius + a];
        const double wb = a + 1 <= radius ? w_host[radius + a + 1] : 0.0;
        const double tot = wa + wb;
        // the point between taps a and a+1 where interpolation mixes them as wa : wb
        offsets[j] = tot != 0.0 ? (a * wa + (a + 1) * wb) / tot : (double)a;
        weights[j] = tot;
    }
    *c0 = w_host[radius];
    *nfetch = j;
    return SHW_OK;
}

shw_status shw_binomial_taps(int32_t ntaps, int32_t drop, double *c0, double *offsets, double *weights,
                             int32_t capacity, int32_t *nfetch)
{
    if (!c0 || !offsets || !weights || !nfetch || ntaps < 1 || ntaps % 2 != 1 || drop < 0) return SHW_EINVAL;
    const int n = ntaps - 1 + 2 * drop;  // b_n = [1, 1] convolved with itself n times
    if (n > 62) return SHW_EUNSUPPORTED;
    uint64_t row[63];
    pascal_row(n, row);
    uint64_t tot = 0;
    for (int k = drop; k <= n - drop; ++k) tot += row[k];
    // the N central taps, renormalised to sum 1
    double w[129];
    const double t = (double)tot;
    for (int k = 0; k < ntaps; ++k) w[k] = (double)row[drop + k] / t;
    return shw_linear_sampling_taps(w, (ntaps - 1) / 2, c0, offsets, weights, capacity, nfetch);
}

}  // extern "C"
