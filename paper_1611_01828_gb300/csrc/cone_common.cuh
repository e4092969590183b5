// Per-entry helpers shared by the eigensolver kernels (cone.cu: Jacobi
// buckets; cone_large.cu: the tridiagonal QR path for larger cliques).
#pragma once

#include <cuda_runtime.h>

namespace hsde {

// The point projected for one packed entry, from the previous s, z, v of
// the entry and gx = (H_k x_hat) of it: a = alpha s_hat + (1-alpha) s - z,
// the new v = alpha v_hat + (1-alpha) v, and hx = (H_k x_new) of it.  alpha
// is uniform over the launch, so the branch does not diverge; alpha = 1
// reads nothing more.  In the clique's precision C: s, z, v are stored in
// it and a is projected in it; gx is formed in FP64 by the caller (x_w and
// eta x_p can nearly cancel).  On this GPU FP64 runs at 1/64 of the FP32
// rate, so the mixed form keeps these per-entry terms off the FP64 pipe.
template <typename C>
__device__ __forceinline__ void cone_inputs(C so, C zo, C vo, C gx, C al, const double* __restrict__ x, int gi,
                                            C& av, C& vn, C& hx) {
    if (al == C(1)) {
        av = C(0.5) * (so - zo - vo + gx);
        vn = C(0.5) * (so + zo + vo - gx);
        hx = gx;
    } else {
        const C sh = C(0.5) * (so + zo - vo + gx);
        av = al * sh + (C(1) - al) * so - zo;
        vn = al * C(0.5) * (so + zo + vo - gx) + (C(1) - al) * vo;
        hx = al * gx + (C(1) - al) * (C)x[gi];
    }
}

// Column of entry e in a packed lower column-major c x c block (column b
// starts at b c - b (b - 1) / 2).
__device__ __forceinline__ int packed_column(int e, int c) {
    const float cc = 2.f * c + 1.f;
    int b = (int)((cc - sqrtf(fmaxf(cc * cc - 8.f * e, 0.f))) * 0.5f);
    b = max(0, min(b, c - 1));
    while (b > 0 && b * c - b * (b - 1) / 2 > e) --b;
    while (b + 1 < c && (b + 1) * c - (b + 1) * b / 2 <= e) ++b;
    return b;
}

}  // namespace hsde
