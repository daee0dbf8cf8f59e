// Register-level pieces of the z transforms shared by the spectral kernels: the padded shared-memory
// layout of a column, multiplication by -+i, and the small in-register DFTs (radix 2, 4, 8).
#pragma once
#include "common.cuh"

namespace fdetd {

// Shared-memory layout of one column: element p at pad16(p) = p + 2 floor(p / 16), two pad slots
// after every 16 elements, so 16-byte pairs stay aligned for the asynchronous copies and the strided
// butterflies of every stage fall on distinct banks.
__host__ __device__ __forceinline__ constexpr int pad16(int p) { return p + ((p >> 4) << 1); }

// multiply by -i (forward) / +i (inverse)
template <bool INV, typename C>
__device__ __forceinline__ C rot90(C a) {
  C r;
  if (INV) {
    r.x = -a.y;
    r.y = a.x;
  } else {
    r.x = a.y;
    r.y = -a.x;
  }
  return r;
}

// In-register DFT of RR points, natural order in and out (W = exp(-+2 pi i / RR)).
template <int RR, bool INV, typename C>
__device__ __forceinline__ void dft_small(C* v) {
  if (RR == 2) {
    const C t = v[1];
    v[1] = csub(v[0], t);
    v[0] = cadd(v[0], t);
  } else if (RR == 4) {
    const C a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]), a2 = cadd(v[1], v[3]);
    const C a3 = rot90<INV>(csub(v[1], v[3]));
    v[0] = cadd(a0, a2);
    v[2] = csub(a0, a2);
    v[1] = cadd(a1, a3);
    v[3] = csub(a1, a3);
  } else {  // 8: two 4-point DFTs (even / odd samples) and one radix-2 stage
    C e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft_small<4, INV>(e);
    dft_small<4, INV>(o);
    typedef decltype(e[0].x) R;
    const R h = (R)0.70710678118654752440;
    C w1, w3;  // W8^1, W8^3 (forward), conjugates for the inverse
    w1.x = h;
    w1.y = INV ? h : -h;
    w3.x = -h;
    w3.y = INV ? h : -h;
    const C t0 = o[0], t1 = cmul(w1, o[1]), t2 = rot90<INV>(o[2]), t3 = cmul(w3, o[3]);
    v[0] = cadd(e[0], t0);
    v[4] = csub(e[0], t0);
    v[1] = cadd(e[1], t1);
    v[5] = csub(e[1], t1);
    v[2] = cadd(e[2], t2);
    v[6] = csub(e[2], t2);
    v[3] = cadd(e[3], t3);
    v[7] = csub(e[3], t3);
  }
}

}  // namespace fdetd
