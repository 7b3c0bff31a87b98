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
// inverse runs the same steps backwards from those registers, so a pass with an
// operator between the two transforms (the z passes: Eq. 13, Eq. 20) touches
// shared memory only for two transposes per component, against twelve
// round trips of a block-wide Stockham tile.
//
// A block holds W consecutive kx columns (W x 8 bytes = 128 bytes of a row per
// warp access: W = 16 in FP32, 8 in FP64) and TL threads per column; thread
// (col, t) = (tid % W, tid / W). Global loads and stores of a fixed m (or k)
// are W-column row segments, coalesced. The transposes alternate between two
// buffers, so one __syncthreads per transform suffices. When n2/2 and the
// number of pencils are multiples of W, the lone Nyquist column kx = n2/2 of W
// consecutive pencils shares one extra block (lane column `col` then takes
// pencil outer0 + col), instead of a block with one busy column per pencil.
// All components a thread transforms are requested from global memory before
// the first transform, so a block keeps its loads in flight while it computes.
#pragma once
#include "acm_fft.cuh"
#include "acm_types.h"

namespace acm {

// columns per block of the default register-resident variant: one 128-byte
// row segment per warp access (16 in FP32, 8 in FP64); the narrow variant
// takes half of that
template <typename T>
__host__ __device__ constexpr int rr_wdef() { return 128 / (int)sizeof(cx<T>); }

// NST: operator-state values per element a z pass prefetches (2 Stokes: q^ and
// div^; 1 solute: chi^; 0 for the y passes)
template <typename T, int N, int W, int NST = 0>
struct RCfg {
  static constexpr int TL = N / 16;                        // threads per line
  static constexpr int NT = W * TL;                        // threads per block
  static constexpr int BS = N + 1;                         // column stride of a transpose buffer (odd)
  static constexpr int SMEM = (2 * W * BS + N + NST * 16 * NT) * (int)sizeof(cx<T>);
};

template <int OP>
__host__ __device__ constexpr int rr_nst() { return OP == OP_STOKES ? 2 : (OP == OP_SOLUTE ? 1 : 0); }

// W_N^{e} (forward sign) or its conjugate, e taken modulo N
template <typename T, int N, int SIGN>
__device__ __forceinline__ cx<T> rtw(const cx<T>* tw, int e) {
  cx<T> w = tw[e & (N - 1)];
  if constexpr (SIGN > 0) w.y = -w.y;
  return w;
}

// Forward-ordered half: on entry v[m] = x[t + TL m]; on exit v[i TL + k2] =
// X[k1 + 16 k2] with k1 = t + TL i (the thread now owns k1 = t, t + TL, ...).
template <typename T, int N, int SIGN>
__device__ __forceinline__ void rr_fft(cx<T> (&v)[16], cx<T>* buf, const cx<T>* tw, int col, int t) {
  constexpr int TL = N / 16, BS = N + 1;
  dft<16, SIGN>(v);
#pragma unroll
  for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], rtw<T, N, SIGN>(tw, t * k1));
  cx<T>* b = buf + col * BS;
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) b[k1 * TL + t] = v[k1];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 16 / TL; ++i) {
#pragma unroll
    for (int tt = 0; tt < TL; ++tt) v[i * TL + tt] = b[(t + TL * i) * TL + tt];
    dft<TL, SIGN>(&v[i * TL]);
  }
}

// Inverse-ordered half: on entry v[i TL + k2] = X[k1 + 16 k2], k1 = s + TL i;
// on exit v[m] = x[s + TL m].
template <typename T, int N, int SIGN>
__device__ __forceinline__ void rr_ifft(cx<T> (&v)[16], cx<T>* buf, const cx<T>* tw, int col, int s) {
  constexpr int TL = N / 16, BS = N + 1;
  cx<T>* b = buf + col * BS;
#pragma unroll
  for (int i = 0; i < 16 / TL; ++i) {
    dft<TL, SIGN>(&v[i * TL]);
    const int k1 = s + TL * i;
#pragma unroll
    for (int tt = 1; tt < TL; ++tt) v[i * TL + tt] = cmul(v[i * TL + tt], rtw<T, N, SIGN>(tw, tt * k1));
#pragma unroll
    for (int tt = 0; tt < TL; ++tt) b[k1 * TL + tt] = v[i * TL + tt];
  }
  __syncthreads();
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) v[k1] = b[k1 * TL + s];
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

// Operators (OP values of the block-wide strided kernel, acm_kernels.cuh):
//   OP_FWD / OP_INV  NC components transformed forward / inverse.
//   OP_FWD_SOL (y)   (tau_0, tau_1, s') in, (tau_0, s' + i d1 tau_1) out.
//   OP_INV_SOL (y)   (a, b) in, inverse transforms of (a, i d1 b, i d2 b) out.
//   OP_STOKES (z)    forward, Eq. 13 per wavevector with the q^ update of Eq. 9
//                    and the Parseval partials of the divergence residuals, inverse.
//   OP_SOLUTE (z)    forward of (tau_0, s''), F^ = s'' + i d0 tau_0, Eq. 20 with
//                    the Parseval partials of Eq. 19, inverse of (i d0 chi^, chi^).
template <typename T, int N, int OP, int NC, int W>
__global__ void __launch_bounds__(RCfg<T, N, W>::NT) k_rstrided(PassArgs<T> a) {
  using C = RCfg<T, N, W, rr_nst<OP>()>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* buf0 = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* buf1 = buf0 + W * C::BS;
  cx<T>* tw = buf1 + W * C::BS;
  // z passes: the operator state of the thread's 16 wavevectors, prefetched
  // with cp.async into slots private to the thread ([value][element][thread])
  cx<T>* stp = tw + N;
  __shared__ double red[4 * 32];
  const int p = blockIdx.z;
  const int col = threadIdx.x % W, t = threadIdx.x / W;
  // the lane column's pencil and kx column: a regular block takes W columns of
  // pencil blockIdx.y; the Nyquist block (blockIdx.x == a.nyq_blk) takes column
  // n2/2 of the W pencils W blockIdx.y .. W blockIdx.y + W - 1
  const bool nyq = (int)blockIdx.x == a.nyq_blk;
  const int outer = nyq ? (int)blockIdx.y * W + col : (int)blockIdx.y;
  const int kx = nyq ? a.Pu - 1 : (int)blockIdx.x * W + col;
  const bool live = !nyq || (int)blockIdx.y * W < a.nouter;
  const bool ok = live && kx < a.Pu;
  if ((a.sprm && a.sprm[p].done) || (a.cprm && a.cprm[p].done)) return;
  if (!live) {
    // a Nyquist block past the last pencil: only its partial sums (zero) exist
    if constexpr (OP == OP_STOKES || OP == OP_SOLUTE)
      if (threadIdx.x < 3) a.part[((long long)p * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x) * 4 +
                                  threadIdx.x] = 0.0;
    return;
  }
  for (int k = threadIdx.x; k < N; k += blockDim.x) tw[k] = a.twg[k * (TW_MAX / N)];
  cx<T>* base = a.spec + p * a.probStride + (long long)outer * a.outerStride + kx;
  cx<T> v[16];
  if constexpr (OP == OP_FWD) {
    // component c + 1 travels while component c is transformed
    cx<T> w[16];
    rr_load_x<T, N>(v, base, a.rowStride, t, ok);
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      cx<T>(&cur)[16] = (c & 1) ? w : v;
      cx<T>(&nxt)[16] = (c & 1) ? v : w;
      if (c + 1 < NC) rr_load_x<T, N>(nxt, base + (c + 1) * a.compStride, a.rowStride, t, ok);
      rr_fft<T, N, -1>(cur, (c & 1) ? buf1 : buf0, tw, col, t);
      rr_store_k<T, N>(cur, base + c * a.compStride, a.rowStride, t, ok);
    }
  } else if constexpr (OP == OP_INV) {
    cx<T> w[16];
    rr_load_k<T, N>(v, base, a.rowStride, t, ok);
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      cx<T>(&cur)[16] = (c & 1) ? w : v;
      cx<T>(&nxt)[16] = (c & 1) ? v : w;
      if (c + 1 < NC) rr_load_k<T, N>(nxt, base + (c + 1) * a.compStride, a.rowStride, t, ok);
      rr_ifft<T, N, +1>(cur, (c & 1) ? buf1 : buf0, tw, col, t);
      rr_store_x<T, N>(cur, base + c * a.compStride, a.rowStride, t, ok);
    }
  } else if constexpr (OP == OP_FWD_SOL) {
    constexpr int TL = N / 16;
    cx<T> w[16];
    rr_load_x<T, N>(v, base, a.rowStride, t, ok);
    rr_load_x<T, N>(w, base + a.compStride, a.rowStride, t, ok);
    __syncthreads();
    rr_fft<T, N, -1>(v, buf0, tw, col, t);
    rr_store_k<T, N>(v, base, a.rowStride, t, ok);
    rr_load_x<T, N>(v, base + 2 * a.compStride, a.rowStride, t, ok);
    rr_fft<T, N, -1>(w, buf1, tw, col, t);
#pragma unroll
    for (int e = 0; e < 16; ++e) w[e] = cscale(mul_i(w[e]), a.sym.d1[rr_krow<TL>(t, e)]);
    rr_fft<T, N, -1>(v, buf0, tw, col, t);
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = v[e] + w[e];
    rr_store_k<T, N>(v, base + a.compStride, a.rowStride, t, ok);
  } else if constexpr (OP == OP_INV_SOL) {
    constexpr int TL = N / 16;
    cx<T> b[16];
    rr_load_k<T, N>(v, base, a.rowStride, t, ok);
    rr_load_k<T, N>(b, base + a.compStride, a.rowStride, t, ok);
    __syncthreads();
    rr_ifft<T, N, +1>(v, buf0, tw, col, t);
    rr_store_x<T, N>(v, base, a.rowStride, t, ok);
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = cscale(mul_i(b[e]), a.sym.d1[rr_krow<TL>(t, e)]);
    rr_ifft<T, N, +1>(v, buf1, tw, col, t);
    rr_store_x<T, N>(v, base + a.compStride, a.rowStride, t, ok);
    rr_ifft<T, N, +1>(b, buf0, tw, col, t);
    // i d2(kx) applied after the (linear) transform: a factor per column
    const T d2 = ok ? a.sym.d2[kx] : (T)0;
#pragma unroll
    for (int m = 0; m < 16; ++m) b[m] = cscale(mul_i(b[m]), d2);
    rr_store_x<T, N>(b, base + 2 * a.compStride, a.rowStride, t, ok);
  } else if constexpr (OP == OP_STOKES || OP == OP_SOLUTE) {
    constexpr int TL = N / 16;
    constexpr int NIN = OP == OP_STOKES ? 3 : 2;
    constexpr int NST = rr_nst<OP>();
    const long long gst = (long long)p * a.compStride + (long long)outer * a.outerStride + kx;
    // (the state of problem p sits at p * S: a.compStride is S)
    cx<T> u[NIN][16];
#pragma unroll
    for (int c = 0; c < NIN; ++c) rr_load_x<T, N>(u[c], base + c * a.compStride, a.rowStride, t, ok);
    // the state travels while the forward transforms run
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const long long gi = gst + (long long)rr_krow<TL>(t, e) * a.rowStride;
      cp_async_pred<(int)sizeof(cx<T>)>(&stp[e * C::NT + threadIdx.x], ok ? &a.st0[gi] : a.st0, ok);
      if constexpr (NST == 2)
        cp_async_pred<(int)sizeof(cx<T>)>(&stp[(16 + e) * C::NT + threadIdx.x], ok ? &a.st1[gi] : a.st1, ok);
    }
    cp_async_commit();
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NIN; ++c) rr_fft<T, N, -1>(u[c], (c & 1) ? buf1 : buf0, tw, col, t);
    const T invV = (T)a.invV;
    const int ky = outer;
    const T d1 = a.sym.d1[ky], l1 = a.sym.l1[ky];
    const T d2 = ok ? a.sym.d2[kx] : (T)0, l2 = ok ? a.sym.l2[kx] : (T)0;
    const T wgt = (kx == 0 || kx == a.nkx) ? (T)1 : (T)2;
    const T l12 = l1 + l2, d12 = d1 * d1 + d2 * d2;
    T acc0 = 0, acc1 = 0, acc2 = 0;
    // the operator state (q^ and div^, or chi^) at the thread's wavevectors:
    // read from the prefetched slots, rewritten in place in global memory
    constexpr int CH = 4;
    cp_async_wait<0>();
    if constexpr (OP == OP_STOKES) {
      const T nu = (T)a.sprm[p].nu, beta = (T)a.sprm[p].psi[1], b = (T)a.sprm[p].psi[2];
#pragma unroll
      for (int e0 = 0; e0 < 16; e0 += CH) {
        cx<T> qs[CH], ds[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) {
          qs[j] = stp[(e0 + j) * C::NT + threadIdx.x];
          ds[j] = stp[(16 + e0 + j) * C::NT + threadIdx.x];
        }
#pragma unroll
        for (int j = 0; j < CH; ++j) {
          const int e = e0 + j, kz = rr_krow<TL>(t, e);
          const long long gi = gst + (long long)kz * a.rowStride;
          const T d0 = a.sym.d0[kz], l0 = a.sym.l0[kz];
          const T L = l0 + l12, dd = d0 * d0 + d12;
          const bool k0 = (kz == 0 && ky == 0 && kx == 0);
          // r = w^ - i d q^ (+ g V at k = 0)
          const cx<T> iq = mul_i(qs[j]);
          cx<T> r0 = u[0][e] - cscale(iq, d0), r1 = u[1][e] - cscale(iq, d1), r2 = u[2][e] - cscale(iq, d2);
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
            acc0 += wgt * cabs2(dv);
            acc1 += wgt * cabs2(ddv);
            acc2 += wgt * cabs2(qn);
          }
          if (k0) {
            a.sprm[p].mean_u[0] = (double)v0.x * a.invV;
            a.sprm[p].mean_u[1] = (double)v1.x * a.invV;
            a.sprm[p].mean_u[2] = (double)v2.x * a.invV;
          }
          u[0][e] = cscale(v0, invV);
          u[1][e] = cscale(v1, invV);
          u[2][e] = cscale(v2, invV);
        }
      }
    } else {
      const T A0 = (T)a.cprm[p].A0, B00 = (T)a.cprm[p].B0[0], B01 = (T)a.cprm[p].B0[1],
              B02 = (T)a.cprm[p].B0[2];
#pragma unroll
      for (int e0 = 0; e0 < 16; e0 += CH) {
        cx<T> cs[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) cs[j] = stp[(e0 + j) * C::NT + threadIdx.x];
#pragma unroll
        for (int j = 0; j < CH; ++j) {
          const int e = e0 + j, kz = rr_krow<TL>(t, e);
          const long long gi = gst + (long long)kz * a.rowStride;
          const T d0 = a.sym.d0[kz], l0 = a.sym.l0[kz];
          const T L = l0 + l12, dd = d0 * d0 + d12;
          const bool k0 = (kz == 0 && ky == 0 && kx == 0);
          // F^ = s^ + i d.tau^ (Eq. 18 in Fourier space); the axis-2 and axis-1
          // terms were added in the x and y passes, u[1] holds s''
          const cx<T> F = u[1][e] + mul_i(cscale(u[0][e], d0));
          // Eq. 20: chi^ = F^ / (i B0.d + A0 L), chi^(0) = 0
          const T dre = A0 * L, dim = B00 * d0 + B01 * d1 + B02 * d2;
          cx<T> chi = mk<T>(0, 0);
          if (!k0 && ok) {
            const T den = (T)1 / (dre * dre + dim * dim);
            chi = mk<T>((F.x * dre + F.y * dim) * den, (F.y * dre - F.x * dim) * den);
          }
          if (ok) {
            const cx<T> dch = chi - cs[j];
            a.st0[gi] = chi;
            acc0 += wgt * cabs2(dch);
            acc1 += wgt * dd * cabs2(dch);
          }
          // i d0 chi^ and chi^, normalised for the inverse transforms
          const cx<T> c1 = cscale(chi, invV);
          u[0][e] = cscale(mul_i(c1), d0);
          u[1][e] = c1;
        }
      }
    }
    double v3[3] = {(double)acc0, (double)acc1, (double)acc2};
    const int nb = gridDim.x * gridDim.y;
    block_sum_store<3>(v3, red, a.part + ((long long)p * nb + blockIdx.y * gridDim.x + blockIdx.x) * 4);
    // the last forward transform used buf[(NIN - 1) & 1]; the sums' barriers
    // separate its reads from the inverse transforms' writes
#pragma unroll
    for (int c = 0; c < NIN; ++c) {
      rr_ifft<T, N, +1>(u[c], ((c + NIN) & 1) ? buf1 : buf0, tw, col, t);
      rr_store_x<T, N>(u[c], base + c * a.compStride, a.rowStride, t, ok);
    }
  }
}

}  // namespace acm
