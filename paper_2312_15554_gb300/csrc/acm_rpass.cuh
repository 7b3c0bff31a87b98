// acm_rpass.cuh -- register-resident strided passes (FFTs along y or z) for
// lines of N = 16 * TL points, TL in {4, 8, 16}.
//
// A line (one kx column of one y or z pencil) is held by TL threads, 16
// complex values each, and transformed by the four-step factorisation
// N = 16 x TL:
//   forward  X[k1 + 16 k2] = sum_t W_TL^{t k2} W_N^{t k1} sum_m x[t + TL m] W_16^{m k1}
//   inverse  x[t + TL m]   = sum_k1 W_16^{-m k1} W_N^{-t k1} sum_k2 W_TL^{-t k2} X[k1 + 16 k2]
// Thread t loads x[t + TL m] (m = 0..15) straight from global memory, takes the
// 16-point DFT over m in registers, applies W_N^{t k1}, and hands the values to
// the thread that owns k1 through ONE shared-memory transpose; that thread
// takes the TL-point DFTs over t and holds X[k] for k = s + TL i + 16 k2. The
// inverse runs the same steps backwards from those registers: a transform
// crosses shared memory once (one transpose), against two round trips of a
// block-wide Stockham line plus the staging of its loads and stores.
//
// A tile is W consecutive kx columns of one pencil (W x 8 bytes of a row per
// access: W = 16, 8 or 4 in FP32), held by W x TL threads; thread (col, t) =
// (tid % W, tid / W). When n2/2 and the number of pencils are multiples of W,
// the lone Nyquist column kx = n2/2 of W consecutive pencils forms one more
// tile (lane column `col` takes pencil W g + col), so no tile carries idle
// columns; the tiles of a problem are numbered regular ones first (pencil-major),
// then the Nyquist tiles, and a z pass writes one partial-sum record per tile.
// The transposes alternate between two buffers, so one __syncthreads per
// transform suffices.
//
// k_rstrided runs one tile per block; its global loads go straight to
// registers, the next component's loads issued before the current component's
// transform. A z pass (an operator between the two transforms: Eq. 13, Eq. 20)
// needs every component of a wavevector at once: it parks each forward-
// transformed component in slots of that component's transpose buffer private
// to the thread, so registers never hold more than two components.
#pragma once
#include "acm_fft.cuh"
#include "acm_types.h"

namespace acm {

// columns per block of the default register-resident variant: one 128-byte
// row segment per warp access (16 in FP32, 8 in FP64); the narrow variant
// takes half of that
template <typename T>
__host__ __device__ constexpr int rr_wdef() { return 128 / (int)sizeof(cx<T>); }

// NIN: input components of a tile
template <int OP, int NC>
__host__ __device__ constexpr int rr_nin() {
  return OP == OP_FWD_SOL ? 3 : (OP == OP_INV_SOL ? 2 : (OP == OP_STOKES ? 3 : (OP == OP_SOLUTE ? 2 : NC)));
}

// shared memory of a block (complex elements): two transpose buffers, the
// twiddles and the per-thread state slots
// Transpose buffers hold element (k1, t) of a column at k1 TL + t, the columns
// N + 1 apart, in the wide tiles (a half-warp spans 16 columns, one thread
// each: conflict-free). In the narrow tiles a half-warp holds two threads of
// each of 8 columns, so there the element sits at k1 TL + ((t + k1) mod TL) (a
// skew by k1) and the columns N + 2 apart: the writes by (column, t) and the
// reads by (column, s) of one access then fall on distinct banks.
template <typename T, int N, int W>
struct RCfg {
  static constexpr int TL = N / 16;                          // threads per line
  static constexpr int NT = W * TL;                          // threads per block
  static constexpr bool SKEW = W != rr_wdef<T>();            // narrow tile
  static constexpr int BS = N + (SKEW ? 2 : 1);              // column stride of a transpose buffer
  // position of element (k1, t) within its column
  __device__ static __forceinline__ int at(int k1, int t) { return k1 * TL + (SKEW ? ((t + k1) & (TL - 1)) : t); }
};

// shared memory of a block of pass OP (bytes): transpose buffers of W columns
// (two, or in a z pass one per input component, which then holds that
// component's slots) and the twiddles
template <typename T, int N, int OP, int NC, int W>
__host__ __device__ constexpr int rr_smem() {
  return (((OP == OP_STOKES || OP == OP_SOLUTE) ? rr_nin<OP, NC>() : 2) * W * RCfg<T, N, W>::BS + N) *
         (int)sizeof(cx<T>);
}

// The live tiles of one problem: nreg = gxr pencils x column blocks, then (when
// the Nyquist column is packed) nouter / W Nyquist tiles.
struct RTiles {
  int gxr;     // regular column blocks per pencil
  int nouter;  // pencils
  int nyq;     // 1: the Nyquist column is packed into tiles of its own
  int nlive;   // tiles per problem
};

__host__ __device__ inline RTiles rr_tiles(int Pu, int nouter, int W) {
  RTiles r;
  r.nouter = nouter;
  r.nyq = ((Pu - 1) % W == 0 && nouter % W == 0) ? 1 : 0;
  r.gxr = r.nyq ? (Pu - 1) / W : (Pu + W - 1) / W;
  r.nlive = r.gxr * nouter + (r.nyq ? nouter / W : 0);
  return r;
}

// pencil and kx column of lane column `col` in tile r of a problem
__device__ __forceinline__ void rr_tile_lane(const RTiles& tl, int r, int W, int col, int Pu, int* outer, int* kx) {
  const int nreg = tl.gxr * tl.nouter;
  if (r < nreg) {
    *outer = r / tl.gxr;
    *kx = (r % tl.gxr) * W + col;
  } else {
    *outer = (r - nreg) * W + col;
    *kx = Pu - 1;
  }
}

// W_N^{e} (forward sign) or its conjugate, e taken modulo N
template <typename T, int N, int SIGN>
__device__ __forceinline__ cx<T> rtw(const cx<T>* tw, int e) {
  cx<T> w = tw[e & (N - 1)];
  if constexpr (SIGN > 0) w.y = -w.y;
  return w;
}

// Forward-ordered half: on entry v[m] = x[t + TL m]; on exit v[i TL + k2] =
// X[k1 + 16 k2] with k1 = t + TL i (the thread now owns k1 = t, t + TL, ...).
template <typename T, int N, int W, int SIGN>
__device__ __forceinline__ void rr_fft(cx<T> (&v)[16], cx<T>* buf, const cx<T>* tw, int col, int t) {
  constexpr int TL = N / 16, BS = RCfg<T, N, W>::BS;
  dft<16, SIGN>(v);
#pragma unroll
  for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], rtw<T, N, SIGN>(tw, t * k1));
  cx<T>* b = buf + col * BS;
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) b[RCfg<T, N, W>::at(k1, t)] = v[k1];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 16 / TL; ++i) {
    const int k1 = t + TL * i;
#pragma unroll
    for (int tt = 0; tt < TL; ++tt) v[i * TL + tt] = b[RCfg<T, N, W>::at(k1, tt)];
    dft<TL, SIGN>(&v[i * TL]);
  }
}

// Inverse-ordered half: on entry v[i TL + k2] = X[k1 + 16 k2], k1 = s + TL i;
// on exit v[m] = x[s + TL m].
template <typename T, int N, int W, int SIGN>
__device__ __forceinline__ void rr_ifft(cx<T> (&v)[16], cx<T>* buf, const cx<T>* tw, int col, int s) {
  constexpr int TL = N / 16, BS = RCfg<T, N, W>::BS;
  cx<T>* b = buf + col * BS;
#pragma unroll
  for (int i = 0; i < 16 / TL; ++i) {
    dft<TL, SIGN>(&v[i * TL]);
    const int k1 = s + TL * i;
#pragma unroll
    for (int tt = 1; tt < TL; ++tt) v[i * TL + tt] = cmul(v[i * TL + tt], rtw<T, N, SIGN>(tw, tt * k1));
#pragma unroll
    for (int tt = 0; tt < TL; ++tt) b[RCfg<T, N, W>::at(k1, tt)] = v[i * TL + tt];
  }
  __syncthreads();
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) v[k1] = b[RCfg<T, N, W>::at(k1, s)];
  dft<16, SIGN>(v);
}

// row of element e of a thread's k-held values: k = s + TL i + 16 k2, e = i TL + k2
template <int TL>
__device__ __forceinline__ int rr_krow(int s, int e) {
  return s + TL * (e / TL) + 16 * (e % TL);
}

template <typename T, int N>
__device__ __forceinline__ void rr_load_x(cx<T> (&v)[16], const cx<T>* __restrict__ src, long long rowStride, int t,
                                          bool ok) {
  constexpr int TL = N / 16;
#pragma unroll
  for (int m = 0; m < 16; ++m) v[m] = ok ? src[(long long)(t + TL * m) * rowStride] : mk<T>(0, 0);
}

template <typename T, int N>
__device__ __forceinline__ void rr_store_x(const cx<T> (&v)[16], cx<T>* __restrict__ dst, long long rowStride, int t,
                                           bool ok, T scale = (T)1) {
  constexpr int TL = N / 16;
  if (!ok) return;
#pragma unroll
  for (int m = 0; m < 16; ++m) dst[(long long)(t + TL * m) * rowStride] = scale == (T)1 ? v[m] : cscale(v[m], scale);
}

template <typename T, int N>
__device__ __forceinline__ void rr_load_k(cx<T> (&v)[16], const cx<T>* __restrict__ src, long long rowStride, int s,
                                          bool ok) {
  constexpr int TL = N / 16;
#pragma unroll
  for (int e = 0; e < 16; ++e) v[e] = ok ? src[(long long)rr_krow<TL>(s, e) * rowStride] : mk<T>(0, 0);
}

template <typename T, int N>
__device__ __forceinline__ void rr_store_k(const cx<T> (&v)[16], cx<T>* __restrict__ dst, long long rowStride, int s,
                                           bool ok) {
  constexpr int TL = N / 16;
  if (!ok) return;
#pragma unroll
  for (int e = 0; e < 16; ++e) dst[(long long)rr_krow<TL>(s, e) * rowStride] = v[e];
}

// The z-pass operators on slots: component c of the thread's element e sits
// at sl[c][e * NT] (k-ordered, kz = rr_krow(t, e)) and is replaced there by
// the operator's output; the operator state is read from global memory in
// chunks of SCH elements, all loads of a chunk in flight together. par: the
// operator's parameters in T ((nu, beta, b) or (A0, B0)) and 1/V.
template <typename T>
__host__ __device__ constexpr int rz_chunk() { return sizeof(T) == 4 ? 8 : 4; }

template <typename T, int N, int NT>
__device__ __forceinline__ void rz_stokes_op(const PassArgs<T>& a, cx<T>* const (&sl)[3], const T* par, int p, int ky,
                                             int kx, bool ok, int t, T (&acc)[3]) {
  constexpr int TL = N / 16, SCH = rz_chunk<T>();
  const T nu = par[0], beta = par[1], b = par[2], invV = par[4];
  const T d1 = a.sym.d1[ky], l1 = a.sym.l1[ky];
  const T d2 = ok ? a.sym.d2[kx] : (T)0, l2 = ok ? a.sym.l2[kx] : (T)0;
  const T wgt = (kx == 0 || kx == a.nkx) ? (T)1 : (T)2;
  const T l12 = l1 + l2, d12 = d1 * d1 + d2 * d2;
  const long long gst = (long long)p * a.compStride + (long long)ky * a.outerStride + kx;
#pragma unroll
  for (int e0 = 0; e0 < 16; e0 += SCH) {
    cx<T> qs[SCH], ds[SCH];
#pragma unroll
    for (int j = 0; j < SCH; ++j) {
      const long long gi = gst + (long long)rr_krow<TL>(t, e0 + j) * a.rowStride;
      qs[j] = ok ? a.st0[gi] : mk<T>(0, 0);
      ds[j] = ok ? a.st1[gi] : mk<T>(0, 0);
    }
#pragma unroll
    for (int j = 0; j < SCH; ++j) {
      const int e = e0 + j, kz = rr_krow<TL>(t, e);
      const long long gi = gst + (long long)kz * a.rowStride;
      const T d0 = a.sym.d0[kz], l0 = a.sym.l0[kz];
      const T L = l0 + l12, dd = d0 * d0 + d12;
      const bool k0 = (kz == 0 && ky == 0 && kx == 0);
      // r = w^ - i d q^ (+ g V at k = 0)
      const cx<T> iq = mul_i(qs[j]);
      cx<T> r0 = sl[0][e * NT] - cscale(iq, d0), r1 = sl[1][e * NT] - cscale(iq, d1),
            r2 = sl[2][e * NT] - cscale(iq, d2);
      if (k0) {
        const StokesDev& P = a.sprm[p];
        const T Vt = (T)(1.0 / a.invV);
        r0.x += (T)P.g[0] * Vt;
        r1.x += (T)P.g[1] * Vt;
        r2.x += (T)P.g[2] * Vt;
      }
      // Eq. 13: (nu L + b) u^ + beta d (d.u^) = r, solved as
      //   d.u^ = d.r / (c + beta |d|^2),  u^ = (r - beta d (d.u^)) / c,  c = nu L + b
      const T c0 = nu * L + b;
      const T ic0 = (T)1 / c0;
      const cx<T> dr = cscale(r0, d0) + cscale(r1, d1) + cscale(r2, d2);
      const cx<T> du = cscale(dr, (T)1 / (c0 + beta * dd));
      const cx<T> f = cscale(du, beta);
      const cx<T> v0 = cscale(r0 - cscale(f, d0), ic0);
      const cx<T> v1 = cscale(r1 - cscale(f, d1), ic0);
      const cx<T> v2 = cscale(r2 - cscale(f, d2), ic0);
      // div u^ = i d.u^ from the solve; Eq. 9: q^ <- q^ - beta div u^
      const cx<T> dv = mul_i(du);
      const cx<T> qn = qs[j] - cscale(dv, beta);
      if (ok) {
        a.st0[gi] = qn;
        a.st1[gi] = dv;
        const cx<T> ddv = dv - ds[j];
        acc[0] += wgt * cabs2(dv);
        acc[1] += wgt * cabs2(ddv);
        acc[2] += wgt * cabs2(qn);
      }
      if (k0) {
        a.sprm[p].mean_u[0] = (double)v0.x * a.invV;
        a.sprm[p].mean_u[1] = (double)v1.x * a.invV;
        a.sprm[p].mean_u[2] = (double)v2.x * a.invV;
      }
      sl[0][e * NT] = cscale(v0, invV);
      sl[1][e * NT] = cscale(v1, invV);
      sl[2][e * NT] = cscale(v2, invV);
    }
  }
}

// F^ = s'' + i d0 tau_0, Eq. 20 with chi^(0) = 0, the Parseval partials of
// Eq. 19; the slots leave as (i d0 chi^, chi^) / V.
template <typename T, int N, int NT>
__device__ __forceinline__ void rz_solute_op(const PassArgs<T>& a, cx<T>* const (&sl)[2], const T* par, int p, int ky,
                                             int kx, bool ok, int t, T (&acc)[3]) {
  constexpr int TL = N / 16, SCH = rz_chunk<T>();
  const T A0 = par[0], B00 = par[1], B01 = par[2], B02 = par[3], invV = par[4];
  const T d1 = a.sym.d1[ky], l1 = a.sym.l1[ky];
  const T d2 = ok ? a.sym.d2[kx] : (T)0, l2 = ok ? a.sym.l2[kx] : (T)0;
  const T wgt = (kx == 0 || kx == a.nkx) ? (T)1 : (T)2;
  const T l12 = l1 + l2, d12 = d1 * d1 + d2 * d2;
  const long long gst = (long long)p * a.compStride + (long long)ky * a.outerStride + kx;
#pragma unroll
  for (int e0 = 0; e0 < 16; e0 += SCH) {
    cx<T> cs[SCH];
#pragma unroll
    for (int j = 0; j < SCH; ++j)
      cs[j] = ok ? a.st0[gst + (long long)rr_krow<TL>(t, e0 + j) * a.rowStride] : mk<T>(0, 0);
#pragma unroll
    for (int j = 0; j < SCH; ++j) {
      const int e = e0 + j, kz = rr_krow<TL>(t, e);
      const long long gi = gst + (long long)kz * a.rowStride;
      const T d0 = a.sym.d0[kz], l0 = a.sym.l0[kz];
      const T L = l0 + l12, dd = d0 * d0 + d12;
      const bool k0 = (kz == 0 && ky == 0 && kx == 0);
      const cx<T> F = sl[1][e * NT] + mul_i(cscale(sl[0][e * NT], d0));
      const T dre = A0 * L, dim = B00 * d0 + B01 * d1 + B02 * d2;
      cx<T> chi = mk<T>(0, 0);
      if (!k0 && ok) {
        const T den = (T)1 / (dre * dre + dim * dim);
        chi = mk<T>((F.x * dre + F.y * dim) * den, (F.y * dre - F.x * dim) * den);
      }
      if (ok) {
        const cx<T> dch = chi - cs[j];
        a.st0[gi] = chi;
        acc[0] += wgt * cabs2(dch);
        acc[1] += wgt * dd * cabs2(dch);
      }
      const cx<T> c1 = cscale(chi, invV);
      sl[0][e * NT] = cscale(mul_i(c1), d0);
      sl[1][e * NT] = c1;
    }
  }
}

// Operators (OP values of the block-wide strided kernel, acm_kernels.cuh):
//   OP_FWD / OP_INV  NC components transformed forward / inverse.
//   OP_FWD_SOL (y)   (tau_0, tau_1, s') in, (tau_0, s' + i d1 tau_1) out.
//   OP_INV_SOL (y)   (a, b) in, inverse transforms of (a, i d1 b, i d2 b) out.
//   OP_STOKES (z)    forward, Eq. 13 per wavevector with the q^ update of Eq. 9
//                    and the Parseval partials of the divergence residuals, inverse.
//   OP_SOLUTE (z)    forward of (tau_0, s''), F^ = s'' + i d0 tau_0, Eq. 20 with
//                    the Parseval partials of Eq. 19, inverse of (i d0 chi^, chi^).
// One tile per block (blockIdx.x = problem x live tiles + tile); inputs loaded
// from global memory straight into registers; a z pass writes one partial-sum
// record per tile.
template <typename T, int N, int OP, int NC, int W>
__device__ __forceinline__ void rr_pass_body(const PassArgs<T>& a) {
  using C = RCfg<T, N, W>;
  constexpr int NIN = rr_nin<OP, NC>();
  constexpr bool ZOP = OP == OP_STOKES || OP == OP_SOLUTE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* buf0 = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* buf1 = buf0 + W * C::BS;
  // twiddles after the buffers: NIN of them in a z pass, two otherwise
  cx<T>* tw = buf0 + (ZOP ? NIN : 2) * W * C::BS;
  __shared__ T red[4 * 32];
  __shared__ T opar[5];
  const RTiles tl = rr_tiles(a.Pu, a.nouter, W);
  const int p = blockIdx.x / tl.nlive, r = blockIdx.x % tl.nlive;
  if ((a.sprm && a.sprm[p].done) || (a.cprm && a.cprm[p].done)) return;
  const int col = threadIdx.x % W, t = threadIdx.x / W;
  int outer, kx;
  rr_tile_lane(tl, r, W, col, a.Pu, &outer, &kx);
  const bool ok = kx < a.Pu;
  for (int k = threadIdx.x; k < N; k += blockDim.x) tw[k] = a.twg[k * (TW_MAX / N)];
  if constexpr (ZOP) {
    // the operator's parameters, converted once per block
    if (threadIdx.x == 0) {
      if constexpr (OP == OP_STOKES) {
        opar[0] = (T)a.sprm[p].nu;
        opar[1] = (T)a.sprm[p].psi[1];
        opar[2] = (T)a.sprm[p].psi[2];
      } else {
        opar[0] = (T)a.cprm[p].A0;
        for (int k = 0; k < 3; ++k) opar[1 + k] = (T)a.cprm[p].B0[k];
      }
      opar[4] = (T)a.invV;
    }
  }
  cx<T>* base = a.spec + p * a.probStride + (long long)outer * a.outerStride + kx;
  if constexpr (ZOP) {
    // One component at a time: forward transform in registers (the next
    // component's loads in flight), its k-ordered values parked in slots of its
    // own buffer private to the thread (sl[c][e * NT]); the operator reads and
    // rewrites the slots element by element; then one inverse transform at a
    // time through the same buffers. Registers hold two components at most.
    constexpr int NT = C::NT;
    cx<T>* sl[NIN];
#pragma unroll
    for (int c = 0; c < NIN; ++c) sl[c] = buf0 + c * W * C::BS + threadIdx.x;
    cx<T> v[16], w[16];
    rr_load_x<T, N>(v, base, a.rowStride, t, ok);
    __syncthreads();  // twiddles and parameters
#pragma unroll
    for (int c = 0; c < NIN; ++c) {
      cx<T>(&cur)[16] = (c & 1) ? w : v;
      cx<T>(&nxt)[16] = (c & 1) ? v : w;
      if (c + 1 < NIN) rr_load_x<T, N>(nxt, base + (c + 1) * a.compStride, a.rowStride, t, ok);
      cx<T>* bc = buf0 + c * W * C::BS;
      rr_fft<T, N, W, -1>(cur, bc, tw, col, t);
      __syncthreads();  // every thread has read its transposed values from bc
#pragma unroll
      for (int e = 0; e < 16; ++e) sl[c][e * NT] = cur[e];
    }
    T acc[3] = {(T)0, (T)0, (T)0};
    if constexpr (OP == OP_STOKES) rz_stokes_op<T, N, NT>(a, sl, opar, p, outer, kx, ok, t, acc);
    else rz_solute_op<T, N, NT>(a, sl, opar, p, outer, kx, ok, t, acc);
    block_sum_store<3>(acc, red, a.part + ((long long)p * tl.nlive + r) * 4);
#pragma unroll
    for (int c = 0; c < NIN; ++c) {
      cx<T>* bc = buf0 + c * W * C::BS;
#pragma unroll
      for (int e = 0; e < 16; ++e) v[e] = sl[c][e * NT];
      __syncthreads();  // every thread holds its slots of c before bc is a transpose buffer again
      rr_ifft<T, N, W, +1>(v, bc, tw, col, t);
      rr_store_x<T, N>(v, base + c * a.compStride, a.rowStride, t, ok);
    }
  } else if constexpr (OP == OP_FWD || OP == OP_INV) {
    // component c + 1 travels while component c is transformed
    cx<T> v[16], w[16];
    if constexpr (OP == OP_FWD) rr_load_x<T, N>(v, base, a.rowStride, t, ok);
    else rr_load_k<T, N>(v, base, a.rowStride, t, ok);
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      cx<T>(&cur)[16] = (c & 1) ? w : v;
      cx<T>(&nxt)[16] = (c & 1) ? v : w;
      if (c + 1 < NC) {
        if constexpr (OP == OP_FWD) rr_load_x<T, N>(nxt, base + (c + 1) * a.compStride, a.rowStride, t, ok);
        else rr_load_k<T, N>(nxt, base + (c + 1) * a.compStride, a.rowStride, t, ok);
      }
      if constexpr (OP == OP_FWD) {
        rr_fft<T, N, W, -1>(cur, (c & 1) ? buf1 : buf0, tw, col, t);
        rr_store_k<T, N>(cur, base + c * a.compStride, a.rowStride, t, ok);
      } else {
        rr_ifft<T, N, W, +1>(cur, (c & 1) ? buf1 : buf0, tw, col, t);
        rr_store_x<T, N>(cur, base + c * a.compStride, a.rowStride, t, ok);
      }
    }
  } else if constexpr (OP == OP_FWD_SOL) {
    constexpr int TL = N / 16;
    cx<T> v[16], w[16];
    rr_load_x<T, N>(v, base, a.rowStride, t, ok);
    rr_load_x<T, N>(w, base + a.compStride, a.rowStride, t, ok);
    __syncthreads();
    rr_fft<T, N, W, -1>(v, buf0, tw, col, t);
    rr_store_k<T, N>(v, base, a.rowStride, t, ok);
    rr_load_x<T, N>(v, base + 2 * a.compStride, a.rowStride, t, ok);
    rr_fft<T, N, W, -1>(w, buf1, tw, col, t);
#pragma unroll
    for (int e = 0; e < 16; ++e) w[e] = cscale(mul_i(w[e]), a.sym.d1[rr_krow<TL>(t, e)]);
    rr_fft<T, N, W, -1>(v, buf0, tw, col, t);
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = v[e] + w[e];
    rr_store_k<T, N>(v, base + a.compStride, a.rowStride, t, ok);
  } else {
    // OP_INV_SOL: both inputs in registers first
    constexpr int TL = N / 16;
    static_assert(OP == OP_INV_SOL, "inverse solute pass");
    cx<T> v[16], w[16];
    rr_load_k<T, N>(v, base, a.rowStride, t, ok);
    rr_load_k<T, N>(w, base + a.compStride, a.rowStride, t, ok);
    __syncthreads();
    rr_ifft<T, N, W, +1>(v, buf0, tw, col, t);
    rr_store_x<T, N>(v, base, a.rowStride, t, ok);
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = cscale(mul_i(w[e]), a.sym.d1[rr_krow<TL>(t, e)]);
    rr_ifft<T, N, W, +1>(v, buf1, tw, col, t);
    rr_store_x<T, N>(v, base + a.compStride, a.rowStride, t, ok);
    rr_ifft<T, N, W, +1>(w, buf0, tw, col, t);
    // i d2(kx) applied after the (linear) transform: a factor per column
    const T d2 = ok ? a.sym.d2[kx] : (T)0;
#pragma unroll
    for (int m = 0; m < 16; ++m) w[m] = cscale(mul_i(w[m]), d2);
    rr_store_x<T, N>(w, base + 2 * a.compStride, a.rowStride, t, ok);
  }
}

// the FP32 passes at W = rr_wdef run two blocks per SM at most (shared memory
// and the register file), so they are given 128 registers a thread
template <typename T, int OP, int W>
__host__ __device__ constexpr bool rr_y_wide() {
  return sizeof(T) == 4 && W == rr_wdef<T>();
}

template <typename T, int N, int OP, int NC, int W>
__global__ void __launch_bounds__(RCfg<T, N, W>::NT) k_rstrided(PassArgs<T> a) {
  rr_pass_body<T, N, OP, NC, W>(a);
}

template <typename T, int N, int OP, int NC, int W>
__global__ void __launch_bounds__(RCfg<T, N, W>::NT, 2) k_rstrided_w(PassArgs<T> a) {
  rr_pass_body<T, N, OP, NC, W>(a);
}

}  // namespace acm
