// acm_xline.cuh -- x passes with line-resident components.
//
// A real line of N2 values along the contiguous axis is transformed as a
// complex line of M = N2/2 values z_j = x_{2j} + i x_{2j+1} (see the pre- and
// post-processing formulas in acm_kernels.cuh). TL = M/E consecutive lanes of
// a warp own one line; lane t of the line holds the E elements
// z[t + TL m], m = 0..E-1, in registers.
//
// With E = 16 and TL > 1 the transform has two Stockham stages (radix E, then
// radix TL). The first stage reads exactly the elements t + TL m of its own
// lane, and the second stage leaves its lane with exactly those positions too,
// so between an inverse and a forward transform the local step of the method
// runs on registers, and the voxels 2k, 2k+1 (k = t + TL m) of every component
// belong to the same lane. Shared memory carries only the exchange between the
// two stages, the pairing of k with M - k in the real-transform pre- and
// post-processing, and the spectrum rows on their way in. A line's lanes sit in
// one warp, so every synchronisation is a __syncwarp of those lanes.
#pragma once

#include "acm_fft.cuh"

namespace acm {

template <typename T, int N2>
struct XL {
  static constexpr int M = N2 / 2;
  static constexpr int E = ept(M);
  static constexpr int TL = M / E;        // lanes per line
  static constexpr int LPW = 32 / TL;     // lines per warp
  static constexpr int NB = E / TL;       // second-stage groups per lane (TL > 1)
  // slots per line buffer: X[0..M] (pad(M) included), bank-friendly for TL lanes
  static constexpr int LS = line_stride(M + 1, TL, 0, wave_slots<T>());
  // stride between the consecutive lines of a warp holding NBUF buffers each:
  // an odd multiple of TL modulo the wavefront, so that the lines of one
  // access fall on different banks
  template <int NBUF>
  __host__ __device__ static constexpr int lb() {
    constexpr int W = wave_slots<T>();
    int s = NBUF * LS;
    if (TL < W)
      while ((s / TL) % 2 == 0 || s % TL != 0) ++s;
    return s;
  }
};

// Indicator bits of the lane's voxels 2k, 2k+1 (k = t + TL m) as bits 2m, 2m+1.
// Hb: one bit per voxel, 32 voxels per word in index order (lines of N2 >= 32
// voxels start on a word); the words of a line are read by all its lanes.
// Shorter lines read the bytes of H.
template <int N2, int TL, int E>
__device__ __forceinline__ unsigned xl_hmask(const uint32_t* __restrict__ Hb, const uint8_t* __restrict__ H,
                                             long long line, int t) {
  unsigned hm = 0;
  if constexpr (N2 >= 32) {
    constexpr int NW = N2 / 32, SPW = 16 / TL;  // values of m per word
    const uint32_t* w = Hb + line * NW;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const unsigned word = __ldg(w + m / SPW);
      hm |= ((word >> (2 * t + 2 * TL * (m % SPW))) & 3u) << (2 * m);
    }
  } else {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const uchar2 h = *reinterpret_cast<const uchar2*>(H + line * N2 + 2 * (t + TL * m));
      hm |= (h.x ? 1u : 0u) << (2 * m) | (h.y ? 1u : 0u) << (2 * m + 1);
    }
  }
  return hm;
}

// Mask of the lanes of a warp that own lines (all of them when the warp is full).
__device__ __forceinline__ unsigned xl_mask() { return 0xffffffffu; }

// Pre- and post-processing twiddles. Lane t of a line holds k = t + TL m, and
// W^k = W^t exp(-2 pi i m / (2E)) with W = exp(-2 pi i / N2), because N2 = 2 E TL:
// the lane reads W^t once and multiplies by compile-time roots.

// Z_k from the half spectrum: (X_k + conj X_{M-k}) + i (X_k - conj X_{M-k}) conj(W^k),
// with wt = W^t and k = t + TL m
template <int m, int E, typename T>
__device__ __forceinline__ cx<T> xl_pre(cx<T> X, cx<T> Y, cx<T> wt) {
  const cx<T> e = X + cconj(Y), o = root_mul<+1, m, 2 * E>(cmul(X - cconj(Y), cconj(wt)));
  return e + mul_i(o);
}

// X_k from Z: (Z_k + conj Z_{M-k})/2 - i W^k (Z_k - conj Z_{M-k})/2  (k = 1..M-1)
template <int m, int E, typename T>
__device__ __forceinline__ cx<T> xl_post(cx<T> Zk, cx<T> Zm, cx<T> wt) {
  const T h = (T)0.5;
  const cx<T> a = cscale(Zk + cconj(Zm), h), b = cscale(Zk - cconj(Zm), h);
  return a - mul_i(root_mul<-1, m, 2 * E>(cmul(wt, b)));
}

// Second Stockham stage (radix TL, span E) between shared memory and v:
// reads positions t + TL i + E r, writes nothing; v[i + NB r] = outputs.
// Its twiddles W_M^{j r} (j = t + TL i) are W_M^{t r} exp(-2 pi i i r / E):
// the lane reads the TL - 1 values of i = 0 and rotates by compile-time roots.
template <typename T, int N2, int SIGN>
__device__ __forceinline__ void xl_stage2(const cx<T>* sl, const cx<T>* tw, int t, cx<T> (&v)[XL<T, N2>::E]) {
  using L = XL<T, N2>;
  constexpr int M = L::M, E = L::E, TL = L::TL, NB = L::NB;
  cx<T> w0[TL];
  const cx<T>* tws = tw + tw_offset(M, E) + t;
#pragma unroll
  for (int r = 1; r < TL; ++r) {
    w0[r] = tws[(r - 1) * E];
    if constexpr (SIGN > 0) w0[r].y = -w0[r].y;
  }
  static_for<NB>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int j = t + TL * i;
    cx<T> w2[TL];
#pragma unroll
    for (int r = 0; r < TL; ++r) w2[r] = sl[pad(j + E * r)];
    static_for<TL - 1>([&](auto R1) {
      constexpr int r = decltype(R1)::value + 1;
      w2[r] = root_mul<SIGN, i * r, E>(cmul(w2[r], w0[r]));
    });
    dft<TL, SIGN>(w2);
#pragma unroll
    for (int r = 0; r < TL; ++r) v[i + NB * r] = w2[r];
  });
}

// Inverse real transform of one line. sl holds the half spectrum X[0..M]
// (at pad(k)) and is visible to all lanes of the line. On return v[m] =
// z[t + TL m]; sl is free for reuse by the line's lanes.
template <typename T, int N2>
__device__ __forceinline__ void xl_inverse(cx<T>* sl, const cx<T>* tw, int t, unsigned mask,
                                           cx<T> (&v)[XL<T, N2>::E]) {
  using L = XL<T, N2>;
  constexpr int M = L::M, E = L::E, TL = L::TL;
  const cx<T> wt = tw[tw_total(M) + t];
  static_for<E>([&](auto R) {
    constexpr int r = decltype(R)::value;
    const int k = t + TL * r;
    v[r] = xl_pre<r, E>(sl[pad(k)], sl[pad(M - k)], wt);
  });
  dft<E, +1>(v);
  if constexpr (TL > 1) {
    __syncwarp(mask);  // every lane has read its X pairs
#pragma unroll
    for (int r = 0; r < E; ++r) sl[pad(t * E + r)] = v[r];
    __syncwarp(mask);
    xl_stage2<T, N2, +1>(sl, tw, t, v);
    __syncwarp(mask);  // the stage-2 reads are done before sl is reused
  }
}

// Forward real transform of one line: v[m] = z[t + TL m] in; on return
// X[m] = X_{t + TL m} (m = 0..E-1) and, on lane t = 0, xn = X_M (X may be v).
// sl is used as exchange buffer (its previous contents are dropped) and is
// free for the line's lanes on return.
//
// The post-processing pairs Z_k with Z_{M-k}. With k = t + TL m, M - k is
// position E-1-m of lane TL - t when t > 0, and position E - m of lane 0 itself
// when t = 0, so the partners travel by warp shuffles (lane t exchanges with
// lane (TL - t) mod TL of its line) instead of a second pass through sl.
// Positions m and E-1-m are finished together; lane 0's partner E - m of
// position m was overwritten one step earlier and is carried in a register.
template <typename T, int N2>
__device__ __forceinline__ void xl_forward(cx<T>* sl, const cx<T>* tw, int t, unsigned mask,
                                           cx<T> (&v)[XL<T, N2>::E], cx<T> (&X)[XL<T, N2>::E], cx<T>& xn) {
  using L = XL<T, N2>;
  constexpr int M = L::M, E = L::E, TL = L::TL;
  static_assert(E % 2 == 0, "positions finish in pairs");
  const cx<T> wt = tw[tw_total(M) + t];
  dft<E, -1>(v);
  __syncwarp(mask);  // earlier readers of sl are done
#pragma unroll
  for (int r = 0; r < E; ++r) sl[pad(t * E + r)] = v[r];
  if constexpr (TL > 1) {
    __syncwarp(mask);
    xl_stage2<T, N2, -1>(sl, tw, t, v);
    __syncwarp(mask);  // the stage-2 reads are done before sl is reused
  }
  // Z_k sits in v[m] of its own lane
  const int lane = threadIdx.x & 31;
  const int src = (lane - t) + (TL - t) % TL;
  cx<T> carry = mk<T>((T)0, (T)0);
  static_for<E / 2>([&](auto I) {
    constexpr int m = decltype(I)::value, mb = E - 1 - m;
    const cx<T> a = v[m], b = v[mb];
    cx<T> pa, pb;  // the partner lane's v[E-1-m] and v[m]
    pa.x = __shfl_sync(mask, b.x, src);
    pa.y = __shfl_sync(mask, b.y, src);
    pb.x = __shfl_sync(mask, a.x, src);
    pb.y = __shfl_sync(mask, a.y, src);
    // lane 0: Z_{M-k} of position m is its own old v[E-m] (carried; position 0
    // is k = 0), that of position E-1-m its own v[m+1] (b itself when m+1 = E-1-m)
    const cx<T> zm = t == 0 ? carry : pa;
    const cx<T> zb = t == 0 ? (m + 1 == mb ? b : v[m + 1 < E ? m + 1 : 0]) : pb;
    carry = b;
    if (m == 0 && t == 0) {
      X[m] = mk<T>(a.x + a.y, (T)0);
      xn = mk<T>(a.x - a.y, (T)0);
    } else {
      X[m] = xl_post<m, E>(a, zm, wt);
    }
    X[mb] = xl_post<mb, E>(b, zb, wt);
  });
}

}  // namespace acm
