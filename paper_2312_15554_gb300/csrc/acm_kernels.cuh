// acm_kernels.cuh -- the ACM hot path as fused FFT-pass kernels (sm_103a).
//
// One Stokes ADMM iteration (Section 3.1) is five pass kernels plus a tiny
// FP64 finalize kernel:
//   x_stokes_local   C2R along x of u^{n+1}, steps 2-3 (Eq. 8-9) pointwise,
//                    partial sums of the Eq. 10 residuals
//   stokes_finalize  residuals, tolerances (Eq. 11-12), stop test, Eq. 22
//   x_stokes_rhs     w = b u~ - a (the known part of Eq. 7), R2C along x
//   strided<FWD>     forward FFT along y
//   strided<STOKES>  forward FFT along z, Eq. 13 solve per wavevector, q update
//                    of Eq. 9 in Fourier space, divergence residuals by
//                    Parseval, inverse FFT along z
//   strided<INV>     inverse FFT along y
// One solute iteration (Section 3.2) is x_solute (C2R of grad chi, local
// residual terms of Eq. 18, R2C), strided<FWD>, strided<SOLUTE> (Eq. 20 with
// the Eq. 21 symbols, Eq. 19 residuals by Parseval), strided<INV> and
// solute_finalize.
//
// The ADMM state is reduced by an identity of steps 2-3: with a^0 = H lambda^0,
// step 3 gives a^{n+1} = H lambda^{n+1} after every iteration, so a is never
// stored, u~ = u on pore voxels and u~ = b u / (b + alpha) on solid voxels.
// The multiplier q only enters through its gradient and is kept in Fourier space.
#pragma once
#include "acm_fft.cuh"
#include "acm_types.h"

namespace acm {

// ---------------------------------------------------------------------------
// x-pass configuration (real lines of length N2, complex FFT of length M = N2/2)
// ---------------------------------------------------------------------------
template <typename T, int N2>
struct XCfg {
  static constexpr int M = N2 / 2;
  static constexpr int E = ept(M);
  static constexpr int TL = M / E;          // threads per line transform
  static constexpr int LPB = 64 / TL;       // lines per block
  static constexpr int LS = line_stride(M, TL, 0, wave_slots<T>());  // complex slots per component line
};

// dynamic shared memory of an x-pass kernel with NC component lines per line
template <typename T, int N2, int NC>
constexpr int x_smem_bytes() {
  return (NC * XCfg<T, N2>::LPB * XCfg<T, N2>::LS + tw_total(N2 / 2) + N2 / 2 + 1) * (int)sizeof(cx<T>);
}

// Shared-memory layout of an x-pass block: NC component lines, the twiddle
// tables, then (16-byte aligned) NR staged real fields of LPB*N2 values and
// the staged indicator bytes.
template <typename T, int N2, int NC, int NR>
struct XLayout {
  using C = XCfg<T, N2>;
  static constexpr int TOT = C::LPB * N2;
  static constexpr int TW = NC * C::LPB * C::LS;                         // complex offset of the twiddles
  static constexpr int RB = ((TW + tw_total(C::M) + C::M + 1) * (int)sizeof(cx<T>) + 15) / 16 * 16;  // bytes
  static constexpr int HB = RB + NR * TOT * (int)sizeof(T);              // byte offset of H
  static constexpr int QB = (HB + (NR > 0 ? TOT : 0) + 15) / 16 * 16;    // byte offset of the Nyquist bins
  static constexpr int BYTES = QB + NC * C::LPB * (int)sizeof(cx<T>);
};

template <typename T>
__device__ __forceinline__ T& re_at(cx<T>* line, int n) {
  return reinterpret_cast<T*>(&line[pad(n >> 1)])[n & 1];
}

// x-pass twiddles: stage tables of the length-N2/2 transform, then W_N2^k for
// k in [0, N2/2] (real-to-complex post-processing) at tw + tw_total(N2/2)
template <typename T, int N2>
__device__ __forceinline__ void load_tw_x(cx<T>* tw, const cx<T>* __restrict__ twg) {
  FillTw<T, N2 / 2, 1, TW_MAX>::run(tw, twg);
  cx<T>* post = tw + tw_total(N2 / 2);
  for (int k = threadIdx.x; k <= N2 / 2; k += blockDim.x) post[k] = twg[k * (TW_MAX / N2)];
}

// contiguous real segment of n values (n * sizeof(T) a multiple of 16) into shared memory
template <typename T>
__device__ __forceinline__ void stage_real(T* dst, const T* __restrict__ src, int n) {
  constexpr int V = 16 / (int)sizeof(T);
  for (int i = threadIdx.x; i < n / V; i += blockDim.x) cp_async<16>(dst + i * V, src + i * V);
}

// Real transforms of length N2 run as complex transforms of length M = N2/2 on
// z_j = x_{2j} + i x_{2j+1}, with W = exp(-2 pi i / N2):
//   inverse: from the half spectrum X[0..M],
//     Z_k = (X_k + conj X_{M-k}) + i (X_k - conj X_{M-k}) W^{-k},
//     and the unnormalised inverse length-M transform of Z is N2 * z;
//   forward: from Z = forward length-M transform of z,
//     X_k = (Z_k + conj Z_{M-k})/2 - i W^k (Z_k - conj Z_{M-k})/2, k = 0..M (Z_M = Z_0).
//
// x_load_spec_pre: rows of NC half-spectrum components read from global memory
// and turned into Z[0..M-1] on the way into shared memory; each pair (k, M-k)
// is loaded once and written once.
template <typename T, int N2, int NC>
__device__ __forceinline__ void x_load_spec_pre(cx<T>* sm, const cx<T>* __restrict__ spec, long long S, int P,
                                                int line0, const cx<T>* twx) {
  using C = XCfg<T, N2>;
  constexpr int M = C::M;
  const cx<T>* tw = twx + tw_total(M);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int cl = warp; cl < NC * C::LPB; cl += nw) {
    const int c = cl / C::LPB, l = cl - c * C::LPB;
    const cx<T>* src = spec + c * S + (long long)(line0 + l) * P;
    cx<T>* s = sm + cl * C::LS;
    for (int k = lane; k <= M / 2; k += 32) {
      const cx<T> X = src[k], Y = src[M - k];
      const cx<T> e1 = X + cconj(Y), o1 = cmul(X - cconj(Y), cconj(tw[k]));
      const cx<T> e2 = Y + cconj(X), o2 = cmul(Y - cconj(X), cconj(tw[M - k]));
      s[pad(k)] = e1 + mul_i(o1);
      if (k != 0) s[pad(M - k)] = e2 + mul_i(o2);
    }
  }
}

// x_load_spec_raw_async: rows of NC half-spectrum components copied as they are
// (cp.async) into the lines, X[M] into nyq[component line]; x_pre_smem then
// turns them into Z[0..M-1] in place.
template <typename T, int N2, int NC>
__device__ __forceinline__ void x_load_spec_raw_async(cx<T>* sm, cx<T>* nyq, const cx<T>* __restrict__ spec,
                                                      long long S, int P, int line0) {
  using C = XCfg<T, N2>;
  constexpr int M = C::M;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int cl = warp; cl < NC * C::LPB; cl += nw) {
    const int c = cl / C::LPB, l = cl - c * C::LPB;
    const cx<T>* src = spec + c * S + (long long)(line0 + l) * P;
    cx<T>* dst = sm + cl * C::LS;
    for (int k = lane; k < M; k += 32) cp_async<(int)sizeof(cx<T>)>(&dst[pad(k)], &src[k]);
    if (lane == 0) cp_async<(int)sizeof(cx<T>)>(&nyq[cl], &src[M]);
  }
}

// With dc >= 0 the lines of component dc are first multiplied by i d(k)
// (d: the derivative symbol of the kx axis, M + 1 values): they become the
// half spectrum of that component's derivative along the line.
template <typename T, int N2, int NC>
__device__ __forceinline__ void x_pre_smem(cx<T>* sm, const cx<T>* nyq, const cx<T>* twx, int dc = -1,
                                           const T* __restrict__ d = nullptr) {
  using C = XCfg<T, N2>;
  constexpr int M = C::M;
  const cx<T>* tw = twx + tw_total(M);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int cl = warp; cl < NC * C::LPB; cl += nw) {
    cx<T>* s = sm + cl * C::LS;
    const bool der = cl / C::LPB == dc;
    for (int k = lane; k <= M / 2; k += 32) {
      cx<T> X = s[pad(k)], Y = (k == 0) ? nyq[cl] : s[pad(M - k)];
      if (der) {
        X = cscale(mul_i(X), d[k]);
        Y = cscale(mul_i(Y), d[M - k]);
      }
      const cx<T> e1 = X + cconj(Y), o1 = cmul(X - cconj(Y), cconj(tw[k]));
      const cx<T> e2 = Y + cconj(X), o2 = cmul(Y - cconj(X), cconj(tw[M - k]));
      s[pad(k)] = e1 + mul_i(o1);
      if (k != 0) s[pad(M - k)] = e2 + mul_i(o2);
    }
  }
}

// x_post_store_spec: Z[0..M-1] in shared memory -> half spectrum X[0..M]
// written to global memory.
template <typename T, int N2, int NC>
__device__ __forceinline__ void x_post_store_spec(const cx<T>* sm, cx<T>* __restrict__ spec, long long S, int P,
                                                  int line0, const cx<T>* twx) {
  using C = XCfg<T, N2>;
  constexpr int M = C::M;
  const cx<T>* tw = twx + tw_total(M);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const T half = (T)0.5;
  for (int cl = warp; cl < NC * C::LPB; cl += nw) {
    const int c = cl / C::LPB, l = cl - c * C::LPB;
    cx<T>* dst = spec + c * S + (long long)(line0 + l) * P;
    const cx<T>* s = sm + cl * C::LS;
    for (int k = lane; k <= M / 2; k += 32) {
      const cx<T> Zk = s[pad(k)];
      if (k == 0) {
        dst[0] = mk<T>(Zk.x + Zk.y, (T)0);
        dst[M] = mk<T>(Zk.x - Zk.y, (T)0);
      } else {
        const cx<T> Zm = s[pad(M - k)];
        const cx<T> ak = cscale(Zk + cconj(Zm), half), bk = cscale(Zk - cconj(Zm), half);
        const cx<T> am = cscale(Zm + cconj(Zk), half), bm = cscale(Zm - cconj(Zk), half);
        dst[k] = ak - mul_i(cmul(tw[k], bk));
        dst[M - k] = am - mul_i(cmul(tw[M - k], bm));
      }
    }
  }
}

// Solute x-pass output: lines (tau_0, tau_1, tau_2, s) -> half spectra
// (tau_0, tau_1, s + i d2 tau_2) in components 0..2. Adding the axis-2 term of
// i d.tau^ (Eq. 18 in Fourier space) here, where kx is already known, leaves
// three components for the y pass instead of four.
template <typename T, int N2>
__device__ __forceinline__ void x_post_store_solute(const cx<T>* sm, cx<T>* __restrict__ spec, long long S, int P,
                                                    int line0, const cx<T>* twx, const T* __restrict__ d2) {
  using C = XCfg<T, N2>;
  constexpr int M = C::M;
  const cx<T>* tw = twx + tw_total(M);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const T half = (T)0.5;
  // half spectrum value at k (and M - k) of the line in shared memory
  auto post = [&](const cx<T>* s, int k, cx<T>& Xk, cx<T>& Xm) {
    const cx<T> Zk = s[pad(k)];
    if (k == 0) {
      Xk = mk<T>(Zk.x + Zk.y, (T)0);
      Xm = mk<T>(Zk.x - Zk.y, (T)0);
    } else {
      const cx<T> Zm = s[pad(M - k)];
      const cx<T> ak = cscale(Zk + cconj(Zm), half), bk = cscale(Zk - cconj(Zm), half);
      const cx<T> am = cscale(Zm + cconj(Zk), half), bm = cscale(Zm - cconj(Zk), half);
      Xk = ak - mul_i(cmul(tw[k], bk));
      Xm = am - mul_i(cmul(tw[M - k], bm));
    }
  };
  for (int cl = warp; cl < 3 * C::LPB; cl += nw) {
    const int c = cl / C::LPB, l = cl - c * C::LPB;
    cx<T>* dst = spec + c * S + (long long)(line0 + l) * P;
    const cx<T>* s = sm + cl * C::LS;
    const cx<T>* s3 = sm + (3 * C::LPB + l) * C::LS;
    for (int k = lane; k <= M / 2; k += 32) {
      cx<T> Xk, Xm;
      post(s, k, Xk, Xm);
      if (c == 2) {
        cx<T> Sk, Sm;
        post(s3, k, Sk, Sm);
        Xk = Sk + cscale(mul_i(Xk), d2[k]);
        Xm = Sm + cscale(mul_i(Xm), d2[M - k]);
      }
      dst[k] = Xk;
      dst[M - k] = Xm;
    }
  }
}

// complex FFT of length M on NC * LPB component lines, TL threads per line
template <typename T, int N2, int NC, int SIGN>
__device__ __forceinline__ void x_fft(cx<T>* sm, const cx<T>* tw) {
  using C = XCfg<T, N2>;
  const int job = threadIdx.x / C::TL;
  const unsigned mask = __ballot_sync(0xffffffffu, job < NC * C::LPB);
  if (job < NC * C::LPB) fft_line<T, C::M, SIGN>(sm + job * C::LS, threadIdx.x % C::TL, tw, mask);
}

// ---------------------------------------------------------------------------
// Stokes x-pass 1: C2R of u^{n+1}, steps 2-3 of ADMM, residual partial sums
//
// The block's spectrum rows, u^n and H are staged into shared memory with
// asynchronous copies; H lambda^n is then staged for the solid voxels only,
// overlapping the inverse transform. The local step reads shared memory only.
// ---------------------------------------------------------------------------
template <typename T, int N2>
__global__ void __launch_bounds__(3 * 64) k_x_stokes_local(const cx<T>* __restrict__ spec, T* __restrict__ u,
                                                          T* __restrict__ lam, const uint8_t* __restrict__ H,
                                                          StokesDev* __restrict__ prm, double* __restrict__ part,
                                                          Geo g, const cx<T>* __restrict__ twg) {
  using C = XCfg<T, N2>;
  using Lay = XLayout<T, N2, 3, 6>;
  constexpr int TOT = Lay::TOT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = sm + Lay::TW;
  T* su = reinterpret_cast<T*>(smem_raw + Lay::RB);   // [3][TOT] u^n
  T* sl = su + 3 * TOT;                                // [3][TOT] H lambda^n
  uint8_t* sh = smem_raw + Lay::HB;                    // [TOT] H
  __shared__ double red[5 * 32];
  const int p = blockIdx.y;
  StokesDev* P = prm + p;
  if (P->done) return;
  const T alpha = (T)P->psi[0], b = (T)P->psi[2];
  // u~^n on solid voxels = s_prev u^n (s_prev = 1 before the first iteration)
  const T s_prev = (T)(P->psi_prev[2] / (P->psi_prev[2] + P->psi_prev[0]));
  const T s_now = b / (b + alpha);
  const int line0 = blockIdx.x * C::LPB;
  const long long v0 = (long long)line0 * N2;
  const cx<T>* sp = spec + (long long)p * 3 * g.S;
  T* up = u + (long long)p * 3 * g.V;
  T* lp = lam + (long long)p * 3 * g.V;
  const uint8_t* Hp = H + (long long)(p / g.lph) * g.hs;
  cx<T>* nyq = reinterpret_cast<cx<T>*>(smem_raw + Lay::QB);
  x_load_spec_raw_async<T, N2, 3>(sm, nyq, sp, g.S, g.P, line0);
#pragma unroll
  for (int c = 0; c < 3; ++c) stage_real(su + c * TOT, up + c * g.V + v0, TOT);
  for (int i = threadIdx.x; i < TOT / 16; i += blockDim.x) cp_async<16>(sh + 16 * i, Hp + v0 + 16 * i);
  cp_async_commit();
  load_tw_x<T, N2>(tw, twg);
  cp_async_wait<0>();
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * TOT; i += blockDim.x) {
    const int c = i / TOT, e = i - c * TOT;
    cp_async_pred<(int)sizeof(T)>(sl + i, lp + c * g.V + v0 + e, sh[e] != 0);
  }
  cp_async_commit();
  x_pre_smem<T, N2, 3>(sm, nyq, tw);
  __syncthreads();
  x_fft<T, N2, 3, +1>(sm, tw);
  cp_async_wait<0>();
  __syncthreads();
  T a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
  for (int idx = threadIdx.x; idx < TOT; idx += blockDim.x) {
    const int l = idx / N2, n = idx & (N2 - 1);
    const bool solid = sh[idx] != 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T u1 = re_at(sm + (c * C::LPB + l) * C::LS, n);
      const T u0 = su[c * TOT + idx];
      up[c * g.V + v0 + idx] = u1;
      const T du = u1 - u0;
      a3 += du * du;
      if (solid) {
        const T ut1 = s_now * u1;                 // step 2 (Eq. 8) with a^n = H lambda^n
        const T ut0 = s_prev * u0;
        const T l1 = sl[c * TOT + idx] + alpha * ut1;  // step 3 (Eq. 9)
        lp[c * g.V + v0 + idx] = l1;
        const T dut = ut1 - ut0, dd = u1 - ut1;
        a0 += ut1 * ut1;
        a1 += dut * dut;
        a2 += dd * dd;
        a4 += l1 * l1;
      }
    }
  }
  double v5[5] = {(double)a0, (double)a1, (double)a2, (double)a3, (double)a4};
  block_sum_store<5>(v5, red, part + ((long long)p * gridDim.x + blockIdx.x) * 8);
}

// ---------------------------------------------------------------------------
// Stokes x-pass 2: w = b u~ - a (Eq. 7 right-hand side), R2C along x
// ---------------------------------------------------------------------------
template <typename T, int N2>
__global__ void __launch_bounds__(3 * 64) k_x_stokes_rhs(cx<T>* __restrict__ spec, const T* __restrict__ u,
                                                        const T* __restrict__ lam, const uint8_t* __restrict__ H,
                                                        const StokesDev* __restrict__ prm, Geo g,
                                                        const cx<T>* __restrict__ twg) {
  using C = XCfg<T, N2>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = sm + 3 * C::LPB * C::LS;
  const int p = blockIdx.y;
  const StokesDev* P = prm + p;
  if (P->done) return;
  const T b = (T)P->psi[2];
  const T s_prev = (T)(P->psi_prev[2] / (P->psi_prev[2] + P->psi_prev[0]));
  const int line0 = blockIdx.x * C::LPB;
  cx<T>* sp = spec + (long long)p * 3 * g.S;
  const T* up = u + (long long)p * 3 * g.V;
  const T* lp = lam + (long long)p * 3 * g.V;
  const uint8_t* Hp = H + (long long)(p / g.lph) * g.hs;
  load_tw_x<T, N2>(tw, twg);
  for (int idx = threadIdx.x; idx < C::LPB * N2; idx += blockDim.x) {
    const int l = idx / N2, n = idx & (N2 - 1);
    const long long v = (long long)(line0 + l) * N2 + n;
    const bool solid = Hp[v] != 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T uu = up[c * g.V + v];
      const T w = solid ? b * (s_prev * uu) - lp[c * g.V + v] : b * uu;
      re_at(sm + (c * C::LPB + l) * C::LS, n) = w;
    }
  }
  __syncthreads();
  x_fft<T, N2, 3, -1>(sm, tw);
  __syncthreads();
  x_post_store_spec<T, N2, 3>(sm, sp, g.S, g.P, line0, tw);
}

// ---------------------------------------------------------------------------
// Solute x-pass: C2R of grad chi^n (3 components), local terms of Eq. 18:
//   tau = (A - A0)(grad chi + g),  s = F - (B - B0).(grad chi + g),
//   A = (1 - H) + eta H,  B = Pe (1 - H) u,  F = Pe (1 - H) ubar.g,
// then R2C of (tau_0, tau_1, tau_2, s).
// ---------------------------------------------------------------------------
template <typename T, int N2>
__global__ void __launch_bounds__(4 * 64) k_x_solute(cx<T>* __restrict__ spec, const T* __restrict__ u,
                                                    const uint8_t* __restrict__ H,
                                                    const SoluteDev* __restrict__ prm, Geo g,
                                                    const cx<T>* __restrict__ twg, const T* __restrict__ d2) {
  using C = XCfg<T, N2>;
  using Lay = XLayout<T, N2, 4, 3>;
  constexpr int TOT = Lay::TOT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = sm + Lay::TW;
  T* su = reinterpret_cast<T*>(smem_raw + Lay::RB);   // [3][TOT] u on pore voxels, 0 on solid ones
  uint8_t* sh = smem_raw + Lay::HB;                    // [TOT] H
  const int p = blockIdx.y;
  const SoluteDev* P = prm + p;
  if (P->done) return;
  const T A0 = (T)P->A0, eta = (T)P->eta, Pe = (T)P->Pe, Fc = (T)P->Fc;
  const T g0 = (T)P->g[0], g1 = (T)P->g[1], g2 = (T)P->g[2];
  const T B00 = (T)P->B0[0], B01 = (T)P->B0[1], B02 = (T)P->B0[2];
  const int line0 = blockIdx.x * C::LPB;
  const long long v0 = (long long)line0 * N2;
  cx<T>* sp = spec + (long long)p * 4 * g.S;
  const T* up = u + (long long)p * g.us;
  const uint8_t* Hp = H + (long long)(p / g.lph) * g.hs;
  cx<T>* nyq = reinterpret_cast<cx<T>*>(smem_raw + Lay::QB);
  x_load_spec_raw_async<T, N2, 3>(sm, nyq, sp, g.S, g.P, line0);
  for (int i = threadIdx.x; i < TOT / 16; i += blockDim.x) cp_async<16>(sh + 16 * i, Hp + v0 + 16 * i);
  cp_async_commit();
  load_tw_x<T, N2>(tw, twg);
  cp_async_wait<0>();
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * TOT; i += blockDim.x) {
    const int c = i / TOT, e = i - c * TOT;
    cp_async_pred<(int)sizeof(T)>(su + i, up + c * g.V + v0 + e, sh[e] == 0);
  }
  cp_async_commit();
  // components 0, 1 hold the x spectra of d0 chi and d1 chi, component 2 that of chi
  x_pre_smem<T, N2, 3>(sm, nyq, tw, 2, d2);
  __syncthreads();
  x_fft<T, N2, 3, +1>(sm, tw);
  cp_async_wait<0>();
  __syncthreads();
  for (int idx = threadIdx.x; idx < TOT; idx += blockDim.x) {
    const int l = idx / N2, n = idx & (N2 - 1);
    const bool solid = sh[idx] != 0;
    T& r0 = re_at(sm + (0 * C::LPB + l) * C::LS, n);
    T& r1 = re_at(sm + (1 * C::LPB + l) * C::LS, n);
    T& r2 = re_at(sm + (2 * C::LPB + l) * C::LS, n);
    const T e0 = r0 + g0, e1 = r1 + g1, e2 = r2 + g2;
    const T Am = (solid ? eta : (T)1) - A0;
    T s = B00 * e0 + B01 * e1 + B02 * e2;
    if (!solid) s += Fc - Pe * (su[idx] * e0 + su[TOT + idx] * e1 + su[2 * TOT + idx] * e2);
    r0 = Am * e0;
    r1 = Am * e1;
    r2 = Am * e2;
    re_at(sm + (3 * C::LPB + l) * C::LS, n) = s;
  }
  __syncthreads();
  x_fft<T, N2, 4, -1>(sm, tw);
  __syncthreads();
  x_post_store_solute<T, N2>(sm, sp, g.S, g.P, line0, tw, d2);
}

// ---------------------------------------------------------------------------
// plain x-passes (transforms of NC real components)
// ---------------------------------------------------------------------------
template <typename T, int N2, int NC>
__global__ void __launch_bounds__(NC * 64) k_x_r2c(cx<T>* __restrict__ spec, const T* __restrict__ in, Geo g,
                                                  long long inProbStride, long long specProbStride,
                                                  const cx<T>* __restrict__ twg) {
  using C = XCfg<T, N2>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = sm + NC * C::LPB * C::LS;
  const int p = blockIdx.y;
  const int line0 = blockIdx.x * C::LPB;
  const T* ip = in + p * inProbStride;
  load_tw_x<T, N2>(tw, twg);
  for (int idx = threadIdx.x; idx < NC * C::LPB * N2; idx += blockDim.x) {
    const int n = idx & (N2 - 1), cl = idx / N2;
    const int c = cl / C::LPB, l = cl - c * C::LPB;
    re_at(sm + cl * C::LS, n) = ip[c * g.V + (long long)(line0 + l) * N2 + n];
  }
  __syncthreads();
  x_fft<T, N2, NC, -1>(sm, tw);
  __syncthreads();
  x_post_store_spec<T, N2, NC>(sm, spec + p * specProbStride, g.S, g.P, line0, tw);
}

template <typename T, int N2, int NC>
__global__ void __launch_bounds__(NC * 64) k_x_c2r(const cx<T>* __restrict__ spec, T* __restrict__ out, Geo g,
                                                  long long outProbStride, long long specProbStride,
                                                  const cx<T>* __restrict__ twg) {
  using C = XCfg<T, N2>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = sm + NC * C::LPB * C::LS;
  const int p = blockIdx.y;
  const int line0 = blockIdx.x * C::LPB;
  T* op = out + p * outProbStride;
  load_tw_x<T, N2>(tw, twg);
  __syncthreads();
  x_load_spec_pre<T, N2, NC>(sm, spec + p * specProbStride, g.S, g.P, line0, tw);
  __syncthreads();
  x_fft<T, N2, NC, +1>(sm, tw);
  __syncthreads();
  for (int idx = threadIdx.x; idx < NC * C::LPB * N2; idx += blockDim.x) {
    const int n = idx & (N2 - 1), cl = idx / N2;
    const int c = cl / C::LPB, l = cl - c * C::LPB;
    op[c * g.V + (long long)(line0 + l) * N2 + n] = re_at(sm + cl * C::LS, n);
  }
}

// ---------------------------------------------------------------------------
// strided passes: complex FFTs along y or z on tiles of TX consecutive kx
// columns, with an optional per-wavevector operator between a forward and an
// inverse transform (z-pass only).
// ---------------------------------------------------------------------------
// OP_FWD_SOL (y forward of the solute iteration): lines (tau_0, tau_1, s') in,
//   (tau_0, s' + i d1 tau_1) out.
// OP_SOLUTE (z): (tau_0, s'') in, F^ = s'' + i d0 tau_0, Green step, (i d0 chi^, chi^) out.
// OP_INV_SOL (y inverse): (a, b) in, lines (a, i d1 b, b) inverse-transformed out.
enum { OP_FWD = 0, OP_INV = 1, OP_INV_SCALE = 2, OP_STOKES = 3, OP_SOLUTE = 4, OP_DERIV = 5, OP_FWD_SOL = 6,
       OP_INV_SOL = 7 };

template <typename T>
struct PassArgs {
  cx<T>* spec;
  long long probStride, compStride, rowStride, outerStride;
  int Pu;           // used kx columns
  int n1;           // for wavevector indexing in the z-pass
  Sym<T> sym;
  const cx<T>* twg;
  // operator state
  cx<T>* st0;       // Stokes: q^ ; solute: chi^
  cx<T>* st1;       // Stokes: div^ of the previous iteration
  StokesDev* sprm;
  SoluteDev* cprm;
  double* part;     // per-block partial sums (stride 4 doubles)
  double invV;
  int nkx;          // n2 / 2 (Nyquist column index)
  int dm;           // OP_DERIV: axis of the derivative
};

template <typename T, int N, int OP, int NC, int TX>
struct SCfg {
  static constexpr int E = ept(N);
  static constexpr int TL = N / E;
  static constexpr int LS = line_stride(N, TL, TX, wave_slots<T>());
  static constexpr int JOBS = NC * TX;
  static constexpr int THREADS_ALL = JOBS * TL;
  static constexpr int ROUNDS = THREADS_ALL > 2048 ? 8 : THREADS_ALL > 1024 ? 4 : THREADS_ALL > 512 ? 2 : 1;
  // whole warps only: extra threads take no line but help with loads and stores
  static constexpr int NT = ((THREADS_ALL / ROUNDS) + 31) / 32 * 32;
  static constexpr int SMEM = (NC * TX * LS + tw_total(N)) * (int)sizeof(cx<T>);
};

template <typename T, int N, int OP, int NC, int TX, int SIGN, int NLINES>
__device__ __forceinline__ void s_fft(cx<T>* sm, const cx<T>* tw) {
  using C = SCfg<T, N, OP, NC, TX>;
  constexpr int per_round = C::NT / C::TL;
#pragma unroll 1
  for (int r = 0; r < C::ROUNDS; ++r) {
    const int job = r * per_round + threadIdx.x / C::TL;
    const unsigned mask = __ballot_sync(0xffffffffu, job < NLINES);
    if (job < NLINES) fft_line<T, N, SIGN>(sm + job * C::LS, threadIdx.x % C::TL, tw, mask);
  }
}

template <typename T, int N, int OP, int NC, int TX>
__global__ void __launch_bounds__(SCfg<T, N, OP, NC, TX>::NT) k_strided(PassArgs<T> a) {
  using C = SCfg<T, N, OP, NC, TX>;
  constexpr int NIN = (OP == OP_INV_SOL) ? 2 : NC;
  constexpr int NOUT = (OP == OP_FWD_SOL) ? 2 : NC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = sm + NC * TX * C::LS;
  __shared__ double red[4 * 32];
  const int p = blockIdx.z, outer = blockIdx.y, kx0 = blockIdx.x * TX;
  if (a.sprm && a.sprm[p].done) return;
  if (a.cprm && a.cprm[p].done) return;
  cx<T>* base = a.spec + p * a.probStride + outer * a.outerStride + kx0;
  const int w = min(TX, a.Pu - kx0);
  for (int idx = threadIdx.x; idx < NIN * N * TX; idx += blockDim.x) {
    const int col = idx % TX, j = (idx / TX) % N, c = idx / (TX * N);
    const int line = (OP == OP_INV_SOL && c == 1) ? 2 : c;   // OP_INV_SOL: b goes to line 2
    if (col < w)
      cp_async<(int)sizeof(cx<T>)>(&sm[(line * TX + col) * C::LS + pad(j)],
                                   &base[c * a.compStride + j * a.rowStride + col]);
  }
  cp_async_commit();
  FillTw<T, N, 1, TW_MAX>::run(tw, a.twg);
  cp_async_wait<0>();
  __syncthreads();
  if constexpr (OP == OP_INV || OP == OP_INV_SCALE || OP == OP_INV_SOL) {
    if constexpr (OP == OP_INV_SOL) {
      // line 1 = i d1(ky) b: the axis-1 derivative of chi before its inverse transform
      for (int idx = threadIdx.x; idx < N * TX; idx += blockDim.x) {
        const int col = idx % TX, j = idx / TX;
        const cx<T> b = sm[(2 * TX + col) * C::LS + pad(j)];
        sm[(1 * TX + col) * C::LS + pad(j)] = cscale(mul_i(b), a.sym.d1[j]);
      }
      __syncthreads();
    }
    if constexpr (OP == OP_INV_SCALE) {
      const T s = (T)a.invV;
      for (int idx = threadIdx.x; idx < NC * N * TX; idx += blockDim.x) {
        const int col = idx % TX, j = (idx / TX) % N, c = idx / (TX * N);
        cx<T>& x = sm[(c * TX + col) * C::LS + pad(j)];
        x = cscale(x, s);
      }
      __syncthreads();
    }
    s_fft<T, N, OP, NC, TX, +1, NC * TX>(sm, tw);
  } else {
    s_fft<T, N, OP, NC, TX, -1, NIN * TX>(sm, tw);
  }
  if constexpr (OP == OP_FWD_SOL) {
    // s'' = s' + i d1(ky) tau_1 into line 1
    __syncthreads();
    for (int idx = threadIdx.x; idx < N * TX; idx += blockDim.x) {
      const int col = idx % TX, j = idx / TX;
      cx<T>& t1 = sm[(1 * TX + col) * C::LS + pad(j)];
      t1 = sm[(2 * TX + col) * C::LS + pad(j)] + cscale(mul_i(t1), a.sym.d1[j]);
    }
  }
  if constexpr (OP == OP_DERIV) {
    __syncthreads();
    const T invV = (T)a.invV;
    for (int idx = threadIdx.x; idx < NC * N * TX; idx += blockDim.x) {
      const int col = idx % TX, j = (idx / TX) % N, c = idx / (TX * N);
      if (col >= w) continue;
      const T d = a.dm == 0 ? a.sym.d0[j] : (a.dm == 1 ? a.sym.d1[outer] : a.sym.d2[kx0 + col]);
      cx<T>& x = sm[(c * TX + col) * C::LS + pad(j)];
      x = cscale(mul_i(x), d * invV);
    }
    __syncthreads();
    s_fft<T, N, OP, NC, TX, +1, NC * TX>(sm, tw);
  }
  if constexpr (OP == OP_STOKES || OP == OP_SOLUTE) {
    __syncthreads();
    const T invV = (T)a.invV;
    const int ky = outer;
    const T d1 = a.sym.d1[ky], l1 = a.sym.l1[ky];
    T acc0 = 0, acc1 = 0, acc2 = 0;
    // hoisted parameters of the operator
    T nu = 0, beta = 0, b = 0, A0 = 0, B00 = 0, B01 = 0, B02 = 0;
    if constexpr (OP == OP_STOKES) {
      nu = (T)a.sprm[p].nu;
      beta = (T)a.sprm[p].psi[1];
      b = (T)a.sprm[p].psi[2];
    } else {
      A0 = (T)a.cprm[p].A0;
      B00 = (T)a.cprm[p].B0[0];
      B01 = (T)a.cprm[p].B0[1];
      B02 = (T)a.cprm[p].B0[2];
    }
    // The operator state (q^ and div^, or chi^) is read and rewritten in place:
    // each chunk loads its state before any store (see k_x_stokes_local).
    constexpr int TOT = N * TX, CH = 4;
#pragma unroll 1
    for (int base = 0; base < TOT; base += CH * C::NT) {
      bool ok[CH];
      long long gis[CH];
      cx<T> sa[CH], sb[CH];
#pragma unroll
      for (int k = 0; k < CH; ++k) {
        const int idx = base + k * C::NT + threadIdx.x;
        const int col = idx % TX, j = idx / TX;
        ok[k] = idx < TOT && col < w;
        gis[k] = (long long)p * a.compStride + (long long)j * a.rowStride + (long long)outer * a.outerStride + kx0 + col;
        sa[k] = ok[k] ? a.st0[gis[k]] : mk<T>(0, 0);
        if constexpr (OP == OP_STOKES) sb[k] = ok[k] ? a.st1[gis[k]] : mk<T>(0, 0);
      }
#pragma unroll
      for (int k = 0; k < CH; ++k) {
        if (!ok[k]) continue;
        const int idx = base + k * C::NT + threadIdx.x;
        const int col = idx % TX, j = idx / TX, kx = kx0 + col;
        const long long gi = gis[k];
        const T d0 = a.sym.d0[j], l0 = a.sym.l0[j], d2 = a.sym.d2[kx], l2 = a.sym.l2[kx];
        const T L = l0 + l1 + l2, dd = d0 * d0 + d1 * d1 + d2 * d2;
        const T wgt = (kx == 0 || kx == a.nkx) ? (T)1 : (T)2;
        const bool k0 = (j == 0 && ky == 0 && kx == 0);
        cx<T>* s0 = &sm[(0 * TX + col) * C::LS + pad(j)];
        cx<T>* s1 = &sm[(1 * TX + col) * C::LS + pad(j)];
        if constexpr (OP == OP_STOKES) {
          cx<T>* s2 = &sm[(2 * TX + col) * C::LS + pad(j)];
          const cx<T> qh = sa[k];
          const cx<T> dprev = sb[k];
          // r = w^ - i d q^ (+ g V at k = 0)
          const cx<T> iq = mul_i(qh);
          cx<T> r0 = *s0 - cscale(iq, d0), r1 = *s1 - cscale(iq, d1), r2 = *s2 - cscale(iq, d2);
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
          const cx<T> u0 = cscale(r0 - cscale(f, d0), ic0);
          const cx<T> u1 = cscale(r1 - cscale(f, d1), ic0);
          const cx<T> u2 = cscale(r2 - cscale(f, d2), ic0);
          // div u^ = i d.u^ (taken from the solve, free of the cancellation of
          // summing d_c u^_c when beta is large); Eq. 9: q^ <- q^ - beta div u^
          const cx<T> dv = mul_i(du);
          const cx<T> qn = qh - cscale(dv, beta);
          a.st0[gi] = qn;
          a.st1[gi] = dv;
          const cx<T> ddv = dv - dprev;
          acc0 += wgt * cabs2(dv);
          acc1 += wgt * cabs2(ddv);
          acc2 += wgt * cabs2(qn);
          if (k0) {
            a.sprm[p].mean_u[0] = (double)u0.x * a.invV;
            a.sprm[p].mean_u[1] = (double)u1.x * a.invV;
            a.sprm[p].mean_u[2] = (double)u2.x * a.invV;
          }
          *s0 = cscale(u0, invV);
          *s1 = cscale(u1, invV);
          *s2 = cscale(u2, invV);
        } else {
          // F^ = s^ + i d.tau^ (Eq. 18 in Fourier space): the axis-2 and axis-1
          // terms were added in the x and y passes, line 1 holds s''
          const cx<T> F = *s1 + mul_i(cscale(*s0, d0));
          // Eq. 20: chi^ = F^ / (i B0.d + A0 L), chi^(0) = 0
          const T dre = A0 * L, dim = B00 * d0 + B01 * d1 + B02 * d2;
          cx<T> chi = mk<T>(0, 0);
          if (!k0) {
            const T den = (T)1 / (dre * dre + dim * dim);
            chi = mk<T>((F.x * dre + F.y * dim) * den, (F.y * dre - F.x * dim) * den);
          }
          const cx<T> dch = chi - sa[k];
          a.st0[gi] = chi;
          acc0 += wgt * cabs2(dch);
          acc1 += wgt * dd * cabs2(dch);
          // i d0 chi^ and chi^, normalised for the inverse transform (the
          // axis-1 and axis-2 derivatives are taken in the later passes)
          const cx<T> cs = cscale(chi, invV);
          *s0 = cscale(mul_i(cs), d0);
          *s1 = cs;
        }
      }
    }
    double v3[3] = {(double)acc0, (double)acc1, (double)acc2};
    const int nb = gridDim.x * gridDim.y;
    block_sum_store<3>(v3, red, a.part + ((long long)p * nb + blockIdx.y * gridDim.x + blockIdx.x) * 4);
    __syncthreads();
    s_fft<T, N, OP, NC, TX, +1, NOUT * TX>(sm, tw);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < NOUT * N * TX; idx += blockDim.x) {
    const int col = idx % TX, j = (idx / TX) % N, c = idx / (TX * N);
    if (col < w) base[c * a.compStride + j * a.rowStride + col] = sm[(c * TX + col) * C::LS + pad(j)];
  }
}

// ---------------------------------------------------------------------------
// FP64 reductions over real fields
// ---------------------------------------------------------------------------
// sums[p][0..2] = sum u_c ; [3..5] = sum over pore u_c ; [6] = pore voxels.
// FP64 arithmetic is scarce on this GPU: each thread sums chunks of CHK
// elements in the field's precision and folds every chunk into FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_field_sums(const T* __restrict__ u, const uint8_t* __restrict__ H, long long V,
                                                   long long us, long long hs, double* __restrict__ part) {
  constexpr int CHK = 16;
  __shared__ double red[7 * 32];
  const int p = blockIdx.y;
  const T* up = u + (long long)p * us;
  const uint8_t* Hp = H + (long long)p * hs;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; v0 < V; v0 += stride * CHK) {
    T c[7] = {0, 0, 0, 0, 0, 0, 0};
#pragma unroll 4
    for (int k = 0; k < CHK; ++k) {
      const long long v = v0 + k * stride;
      if (v >= V) break;
      const T a = up[v], b = up[V + v], cc = up[2 * V + v];
      c[0] += a;
      c[1] += b;
      c[2] += cc;
      if (Hp[v] == 0) {
        c[3] += a;
        c[4] += b;
        c[5] += cc;
        c[6] += (T)1;
      }
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) acc[k] += (double)c[k];
  }
  block_sum_store<7>(acc, red, part + ((long long)p * gridDim.x + blockIdx.x) * 8);
}

// Eq. 3 contracted with g, and the extended-domain average:
// out[0..2] = sum_pore [g_i + Pe (ubar - u)_i chi + d_i chi]
// out[3..5] = sum_Y A (g_i + d_i chi) + sum_pore Pe (ubar - u)_i chi
template <typename T>
__global__ void __launch_bounds__(256) k_diffusivity(const T* __restrict__ chi, const T* __restrict__ grad,
                                                    const T* __restrict__ u, const uint8_t* __restrict__ H,
                                                    long long V, long long us, long long hs,
                                                    const SoluteDev* __restrict__ prm, double* __restrict__ part) {
  constexpr int CHK = 16;
  __shared__ double red[6 * 32];
  const int p = blockIdx.y;
  const SoluteDev& P = prm[p];
  const T* cp = chi + (long long)p * V;
  const T* gp = grad + (long long)p * 3 * V;
  const T* up = u + (long long)p * us;
  const uint8_t* Hp = H + (long long)p * hs;
  const T Pe = (T)P.Pe, eta = (T)P.eta;
  const T gg[3] = {(T)P.g[0], (T)P.g[1], (T)P.g[2]};
  const T ub[3] = {(T)P.ubar[0], (T)P.ubar[1], (T)P.ubar[2]};
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; v0 < V; v0 += stride * CHK) {
    T c[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll 4
    for (int k = 0; k < CHK; ++k) {
      const long long v = v0 + k * stride;
      if (v >= V) break;
      const T ch = cp[v];
      const bool pore = Hp[v] == 0;
      const T A = pore ? (T)1 : eta;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const T gi = gg[i] + gp[i * V + v];
        const T pe = pore ? Pe * (ub[i] - up[i * V + v]) * ch : (T)0;
        if (pore) c[i] += gi + pe;
        c[3 + i] += A * gi + pe;
      }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] += (double)c[k];
  }
  block_sum_store<6>(acc, red, part + ((long long)p * gridDim.x + blockIdx.x) * 8);
}

// products of three fields f_i (i = load) over the pore voxels:
// out[0..5] = sum_pore f0 f0, f0 f1, f0 f2, f1 f1, f1 f2, f2 f2
template <typename T>
__global__ void __launch_bounds__(256) k_pore_products(const T* __restrict__ f, const uint8_t* __restrict__ H,
                                                      long long V, double* __restrict__ part) {
  constexpr int CHK = 16;
  __shared__ double red[6 * 32];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; v0 < V; v0 += stride * CHK) {
    T c[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll 4
    for (int k = 0; k < CHK; ++k) {
      const long long v = v0 + k * stride;
      if (v >= V) break;
      if (H[v]) continue;
      const T a = f[v], b = f[V + v], d = f[2 * V + v];
      c[0] += a * a;
      c[1] += a * b;
      c[2] += a * d;
      c[3] += b * b;
      c[4] += b * d;
      c[5] += d * d;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] += (double)c[k];
  }
  block_sum_store<6>(acc, red, part + (long long)blockIdx.x * 8);
}

// state conversion between precisions (mixed-precision continuation)
template <typename S, typename D>
__global__ void k_convert(const S* __restrict__ in, D* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (D)in[i];
}

// x (uint8) broadcast multiply: out = H * in for 3 components (warm-start lambda)
template <typename T>
__global__ void k_mask_solid(const T* __restrict__ in, T* __restrict__ out, const uint8_t* __restrict__ H, long long V) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 3 * V; i += (long long)gridDim.x * blockDim.x)
    out[i] = H[i % V] ? in[i] : (T)0;
}

// i d.u^ of a 3-component half spectrum into a 1-component one (warm start div^0)
template <typename T>
__global__ void k_div_spec(const cx<T>* __restrict__ uh, cx<T>* __restrict__ dv, Geo g, Sym<T> sym) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)g.n0 * g.n1 * g.P;
       i += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(i % g.P);
    const long long r = i / g.P;
    const int ky = (int)(r % g.n1), kz = (int)(r / g.n1);
    if (kx >= g.Pu) {
      dv[i] = mk<T>(0, 0);
      continue;
    }
    const cx<T> s = cscale(uh[i], sym.d0[kz]) + cscale(uh[g.S + i], sym.d1[ky]) + cscale(uh[2 * g.S + i], sym.d2[kx]);
    dv[i] = mul_i(s);
  }
}

// spec[c] *= i d2(kx) on the half spectrum of one component per problem
template <typename T>
__global__ void k_mul_id2(cx<T>* __restrict__ spec, long long ps, Geo g, const T* __restrict__ d2) {
  const int p = blockIdx.y;
  cx<T>* sp = spec + (long long)p * ps;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)g.n0 * g.n1 * g.P;
       i += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(i % g.P);
    if (kx < g.Pu) sp[i] = cscale(mul_i(sp[i]), d2[kx]);
  }
}

// Consistent pressure of a warm start: at an ADMM fixed point the divergence of
// the Step 1 equation (Eq. 7 / Eq. 13) gives |d|^2 q^ = i d.a^ for k != 0, and
// q^ = 0 where |d|^2 = 0. ah: 3 components at stride S (unnormalised
// transforms, the scale q^ is kept in).
template <typename T>
__global__ void k_q_from_a(const cx<T>* __restrict__ ah, cx<T>* __restrict__ q, Geo g, Sym<T> sym) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)g.n0 * g.n1 * g.P;
       i += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(i % g.P);
    const long long r = i / g.P;
    const int ky = (int)(r % g.n1), kz = (int)(r / g.n1);
    const T d0 = sym.d0[kz], d1 = sym.d1[ky], d2 = sym.d2[kx < g.Pu ? kx : 0];
    const T dd = d0 * d0 + d1 * d1 + d2 * d2;
    if (kx >= g.Pu || !(dd > (T)0)) {
      q[i] = mk<T>(0, 0);
      continue;
    }
    const cx<T> s = cscale(ah[i], d0) + cscale(ah[g.S + i], d1) + cscale(ah[2 * g.S + i], d2);
    q[i] = cscale(mul_i(s), (T)1 / dd);
  }
}

}  // namespace acm
