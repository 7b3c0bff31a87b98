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
#include "acm_xline.cuh"
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

// complex FFT of length M on NC * LPB component lines, TL threads per line
template <typename T, int N2, int NC, int SIGN>
__device__ __forceinline__ void x_fft(cx<T>* sm, const cx<T>* tw) {
  using C = XCfg<T, N2>;
  const int job = threadIdx.x / C::TL;
  const unsigned mask = __ballot_sync(0xffffffffu, job < NC * C::LPB);
  if (job < NC * C::LPB) fft_line<T, C::M, SIGN>(sm + job * C::LS, threadIdx.x % C::TL, tw, mask);
}

// ---------------------------------------------------------------------------
// Line-resident x passes (acm_xline.cuh): blocks of XS_WARPS warps, each warp
// taking XS_GPW consecutive groups of LPW lines.
// ---------------------------------------------------------------------------
constexpr int XS_WARPS = 8;   // warps per block of the line-resident x passes
constexpr int XS_GPW = 4;     // line groups per warp
constexpr int XS_PCACHE = 4;  // solute x pass: problems whose parameters a block converts once

template <typename T, int N2>
__host__ __device__ constexpr int xs_tw_slots() { return (tw_total(N2 / 2) + N2 / 2 + 1 + 1) / 2 * 2; }

// shared memory: twiddles, NBUF line buffers per line, and ACC real values per lane
template <typename T, int N2, int NBUF, int ACC>
__host__ __device__ constexpr int xs_smem_bytes() {
  return (xs_tw_slots<T, N2>() + XS_WARPS * XL<T, N2>::LPW * XL<T, N2>::template lb<NBUF>()) * (int)sizeof(cx<T>) +
         XS_WARPS * 32 * ACC * (int)sizeof(T);
}

// blocks per problem of the line-resident x passes
__host__ __device__ constexpr int xs_blocks(int lines, int lpw) {
  return (lines / lpw + XS_WARPS * XS_GPW - 1) / (XS_WARPS * XS_GPW);
}

// ---------------------------------------------------------------------------
// Stokes x-pass 1: C2R of u^{n+1}, steps 2-3 of ADMM, residual partial sums
//
// Line-resident: each component of a line is inverse-transformed into
// registers and the local steps run on the lane's voxel pairs 2k, 2k+1 read
// and written as vectors; a chunk of pairs loads its old state before it
// stores, so no store waits for the load of its own address.
// ---------------------------------------------------------------------------
template <typename T, int N2>
__global__ void __launch_bounds__(XS_WARPS * 32, sizeof(T) == 4 ? 2 : 1)
    k_x_stokes_local(const cx<T>* __restrict__ spec, T* __restrict__ u, T* __restrict__ lam,
                     const uint8_t* __restrict__ H, const uint32_t* __restrict__ Hb, StokesDev* __restrict__ prm,
                     double* __restrict__ part, Geo g, const cx<T>* __restrict__ twg) {
  using L = XL<T, N2>;
  constexpr int M = L::M, E = L::E, TL = L::TL, LPW = L::LPW, LS = L::LS;
  constexpr int LB = L::template lb<2>();
  constexpr int CH = E < 4 ? E : 4;  // voxel pairs per load-then-store chunk
  using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* tw = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* lines = tw + xs_tw_slots<T, N2>();
  __shared__ T red[5 * 32];
  __shared__ T kpar[3];
  const int p = blockIdx.y;
  StokesDev* P = prm + p;
  if (P->done) return;
  load_tw_x<T, N2>(tw, twg);
  if (threadIdx.x == 0) {
    // penalties in the kernel's precision, converted once per block;
    // u~^n on solid voxels = s_prev u^n (s_prev = 1 before the first iteration)
    kpar[0] = (T)P->psi[0];
    kpar[1] = (T)P->psi[2];
    kpar[2] = (T)(P->psi_prev[2] / (P->psi_prev[2] + P->psi_prev[0]));
  }
  __syncthreads();
  const T alpha = kpar[0], b = kpar[1];
  const T s_prev = kpar[2];
  const T s_now = b / (b + alpha);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ll = lane / TL, t = lane % TL;
  const unsigned mask = xl_mask();
  cx<T>* b0 = lines + (warp * LPW + ll) * LB;
  cx<T>* b1 = b0 + LS;
  const cx<T>* sp = spec + (long long)p * 3 * g.S;
  T* up = u + (long long)p * 3 * g.V;
  T* lp = lam + (long long)p * 3 * g.V;
  const long long hcell = (long long)(p / g.lph) * g.hs;
  const uint8_t* Hp = H + hcell;
  const uint32_t* Hbp = Hb + hcell / 32;
  // residual partials of the lane over all its lines, in T (a few hundred terms)
  T d5[5] = {0, 0, 0, 0, 0};
  const int ngroups = g.n0 * g.n1 / LPW;
  const int gbase = (blockIdx.x * XS_WARPS + warp) * XS_GPW;
#pragma unroll 1
  for (int gi = 0; gi < XS_GPW; ++gi) {
    const int grp = gbase + gi;
    if (grp >= ngroups) break;
    const long long line = (long long)grp * LPW + ll;
    const long long v0 = line * N2;
    const cx<T>* srow = sp + line * g.P;
    __syncwarp(mask);
    for (int e = t; e <= M; e += TL) {
      cp_async<(int)sizeof(cx<T>)>(&b0[pad(e)], &srow[e]);
      cp_async<(int)sizeof(cx<T>)>(&b1[pad(e)], &srow[g.S + e]);
    }
    cp_async_commit();
    if (lane == 0) {
      // the group's rows of u^n (consecutive lines are contiguous) and the next
      // group's spectrum rows, on their way to L2; H lambda^n is needed on solid
      // voxels only and is left to the predicated loads
      const long long w0 = (long long)grp * LPW * N2;
      constexpr unsigned RB = LPW * N2 * sizeof(T);
#pragma unroll
      for (int c = 0; c < 3; ++c) prefetch_l2(up + c * g.V + w0, RB);
      if (gi + 1 < XS_GPW && grp + 1 < ngroups) {
        const unsigned SB = (unsigned)(LPW * g.P * sizeof(cx<T>));
#pragma unroll
        for (int c = 0; c < 3; ++c) prefetch_l2(sp + c * g.S + (long long)(grp + 1) * LPW * g.P, SB);
      }
    }
    const unsigned hm = xl_hmask<N2, TL, E>(Hbp, Hp, line, t);
    cp_async_wait<0>();
    __syncwarp(mask);
    T a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
    cx<T> v[E];
    static_assert(E % CH == 0, "whole chunks per component");
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
      cx<T>* bc = c == 1 ? b1 : b0;
      T* uc = up + c * g.V + v0;
      T* lc = lp + c * g.V + v0;
      // old state of the component: the first chunk travels during the inverse
      // transform, the second during the first chunk's arithmetic
      T2 ua[CH], la[CH], ub[CH], lb[CH];
      auto load_chunk = [&](int m0, T2 (&uu)[CH], T2 (&ll)[CH]) {
#pragma unroll
        for (int j = 0; j < CH; ++j) {
          const int k = t + TL * (m0 + j);
          uu[j] = *reinterpret_cast<const T2*>(uc + 2 * k);
          if ((hm >> (2 * (m0 + j))) & 3u) {
            ll[j] = *reinterpret_cast<const T2*>(lc + 2 * k);
          } else {
            ll[j].x = (T)0;
            ll[j].y = (T)0;
          }
        }
      };
      auto step_chunk = [&](int m0, const T2 (&u0)[CH], const T2 (&l0)[CH]) {
#pragma unroll
        for (int j = 0; j < CH; ++j) {
          const int m = m0 + j, k = t + TL * m;
          const bool sa = (hm >> (2 * m)) & 1u, sb = (hm >> (2 * m + 1)) & 1u;
          const T u1a = v[m].x, u1b = v[m].y;
          T2 w;
          w.x = u1a;
          w.y = u1b;
          *reinterpret_cast<T2*>(uc + 2 * k) = w;
          const T dua = u1a - u0[j].x, dub = u1b - u0[j].y;
          a3 += dua * dua + dub * dub;
          if (sa | sb) {
            T2 ln = l0[j];
            if (sa) {
              const T ut1 = s_now * u1a, ut0 = s_prev * u0[j].x;   // step 2 (Eq. 8) with a^n = H lambda^n
              ln.x = l0[j].x + alpha * ut1;                          // step 3 (Eq. 9)
              const T dut = ut1 - ut0, dd = u1a - ut1;
              a0 += ut1 * ut1;
              a1 += dut * dut;
              a2 += dd * dd;
              a4 += ln.x * ln.x;
            }
            if (sb) {
              const T ut1 = s_now * u1b, ut0 = s_prev * u0[j].y;
              ln.y = l0[j].y + alpha * ut1;
              const T dut = ut1 - ut0, dd = u1b - ut1;
              a0 += ut1 * ut1;
              a1 += dut * dut;
              a2 += dd * dd;
              a4 += ln.y * ln.y;
            }
            *reinterpret_cast<T2*>(lc + 2 * k) = ln;   // lambda stays 0 on pore voxels
          }
        }
      };
      load_chunk(0, ua, la);
      xl_inverse<T, N2>(bc, tw, t, mask, v);
      if (c == 0) {
        // the row of component 2 into b0, behind components 0 and 1
        __syncwarp(mask);
        for (int e = t; e <= M; e += TL) cp_async<(int)sizeof(cx<T>)>(&b0[pad(e)], &srow[2 * g.S + e]);
        cp_async_commit();
      }
      // rolling: chunk j + 1 travels while chunk j is stepped
#pragma unroll
      for (int j = 0; j < E / CH; ++j) {
        if (j + 1 < E / CH) {
          if (j & 1) load_chunk((j + 1) * CH, ua, la);
          else load_chunk((j + 1) * CH, ub, lb);
        }
        if (j & 1) step_chunk(j * CH, ub, lb);
        else step_chunk(j * CH, ua, la);
      }
      if (c == 1) {
        cp_async_wait<0>();
        __syncwarp(mask);
      }
    }
    d5[0] += a0;
    d5[1] += a1;
    d5[2] += a2;
    d5[3] += a3;
    d5[4] += a4;
  }
  block_sum_store<5>(d5, red, part + ((long long)p * gridDim.x + blockIdx.x) * 8);
}

// ---------------------------------------------------------------------------
// Stokes x-pass 2: w = b u~ - a (Eq. 7 right-hand side), R2C along x
// ---------------------------------------------------------------------------
template <typename T, int N2>
__global__ void __launch_bounds__(XS_WARPS * 32, sizeof(T) == 4 ? 2 : 1)
    k_x_stokes_rhs(cx<T>* __restrict__ spec, const T* __restrict__ u, const T* __restrict__ lam,
                   const uint8_t* __restrict__ H, const uint32_t* __restrict__ Hb, const StokesDev* __restrict__ prm,
                   Geo g, const cx<T>* __restrict__ twg) {
  using L = XL<T, N2>;
  constexpr int M = L::M, E = L::E, TL = L::TL, LPW = L::LPW;
  constexpr int LB = L::template lb<1>();
  constexpr int CH = E < 8 ? E : 8;  // voxel pairs per chunk of loads
  using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* tw = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* lines = tw + xs_tw_slots<T, N2>();
  __shared__ T kpar[2];
  const int p = blockIdx.y;
  const StokesDev* P = prm + p;
  if (P->done) return;
  load_tw_x<T, N2>(tw, twg);
  if (threadIdx.x == 0) {
    // converted once per block; u~^n on solid voxels = s_prev u^n with the
    // penalties of the iteration just taken
    kpar[0] = (T)P->psi[2];
    kpar[1] = (T)(P->psi_prev[2] / (P->psi_prev[2] + P->psi_prev[0]));
  }
  __syncthreads();
  const T b = kpar[0];
  const T s_prev = kpar[1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ll = lane / TL, t = lane % TL;
  const unsigned mask = xl_mask();
  cx<T>* bl = lines + (warp * LPW + ll) * LB;
  cx<T>* sp = spec + (long long)p * 3 * g.S;
  const T* up = u + (long long)p * 3 * g.V;
  const T* lp = lam + (long long)p * 3 * g.V;
  const long long hcell = (long long)(p / g.lph) * g.hs;
  const int ngroups = g.n0 * g.n1 / LPW;
  const int gbase = (blockIdx.x * XS_WARPS + warp) * XS_GPW;
#pragma unroll 1
  for (int gi = 0; gi < XS_GPW; ++gi) {
    const int grp = gbase + gi;
    if (grp >= ngroups) break;
    const long long line = (long long)grp * LPW + ll;
    const long long v0 = line * N2;
    const unsigned hm = xl_hmask<N2, TL, E>(Hb + hcell / 32, H + hcell, line, t);
    cx<T> v[E];
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
      // Eq. 7 right-hand side w = b u~ - a with a = H lambda (the Green step adds g and -i d q)
      const T* uc = up + c * g.V + v0;
      const T* lc = lp + c * g.V + v0;
#pragma unroll
      for (int m0 = 0; m0 < E; m0 += CH) {
        T2 uu[CH], l0[CH];
#pragma unroll
        for (int jj = 0; jj < CH; ++jj) {
          const int k = t + TL * (m0 + jj);
          uu[jj] = *reinterpret_cast<const T2*>(uc + 2 * k);
          if ((hm >> (2 * (m0 + jj))) & 3u) {
            l0[jj] = *reinterpret_cast<const T2*>(lc + 2 * k);
          } else {
            l0[jj].x = (T)0;
            l0[jj].y = (T)0;
          }
        }
#pragma unroll
        for (int jj = 0; jj < CH; ++jj) {
          const int m = m0 + jj;
          const bool sa = (hm >> (2 * m)) & 1u, sb = (hm >> (2 * m + 1)) & 1u;
          v[m] = mk<T>(sa ? b * (s_prev * uu[jj].x) - l0[jj].x : b * uu[jj].x,
                       sb ? b * (s_prev * uu[jj].y) - l0[jj].y : b * uu[jj].y);
        }
      }
      cx<T> xn;
      xl_forward<T, N2>(bl, tw, t, mask, v, v, xn);
      cx<T>* dst = sp + c * g.S + line * g.P;
#pragma unroll
      for (int m = 0; m < E; ++m) dst[t + TL * m] = v[m];
      if (t == 0) dst[M] = xn;
    }
  }
}

// ---------------------------------------------------------------------------
// Solute x-pass: C2R of the gradient of chi^n (3 components), local terms of Eq. 18:
//   tau = (A - A0)(grad chi + g),  s = F - (B - B0).(grad chi + g),
//   A = (1 - H) + eta H,  B = Pe (1 - H) u,  F = Pe (1 - H) ubar.g,
// then R2C of (tau_0, tau_1, tau_2, s), stored as (tau_0, tau_1, s + i d2 tau_2).
// With the central symbols of Eq. 21 (CEN), i d2(kx) is the transform of the
// periodic central difference (f[j+1] - f[j-1]) N2 / 2 along the line, so
// s + D2 tau_2 is formed on the voxels and one R2C replaces two; the
// neighbouring values of tau_2 come from the adjacent lanes by warp shuffles.
//
// Line-resident (acm_xline.cuh): every warp owns LPW lines; their three
// spectrum rows arrive by cp.async, then each component is inverse-transformed
// into registers, turned into tau_c (and its share of s accumulated) on the
// same registers and forward-transformed, without a block-wide barrier.
// ---------------------------------------------------------------------------
template <typename T, int N2, bool CEN>
__global__ void __launch_bounds__(XS_WARPS * 32, sizeof(T) == 4 ? 2 : 1)
    k_x_solute(cx<T>* __restrict__ spec, const T* __restrict__ u, const uint8_t* __restrict__ H,
               const uint32_t* __restrict__ Hb, const SoluteDev* __restrict__ prm, Geo g,
               const cx<T>* __restrict__ twg, const T* __restrict__ d2, int nprob, int gpw) {
  using L = XL<T, N2>;
  constexpr int M = L::M, E = L::E, TL = L::TL, LPW = L::LPW, LS = L::LS;
  constexpr int LB = L::template lb<2>();
  using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* tw = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* lines = tw + xs_tw_slots<T, N2>();
  // s accumulated per lane as voxel pairs: [m][lane] for conflict-free access
  T2* acc = reinterpret_cast<T2*>(lines + XS_WARPS * LPW * LB) + (threadIdx.x >> 5) * 32 * E;
  // Problems that share one velocity and indicator (us = hs = 0, e.g. the three
  // composition loads of a tensor solve) run back to back on the same warp, so
  // each velocity row crosses DRAM once (up to XS_PCACHE problems per block,
  // blockIdx.y numbering the groups); otherwise blockIdx.y is the problem.
  const bool shared = g.us == 0 && g.hs == 0;
  const int pbeg = shared ? blockIdx.y * XS_PCACHE : blockIdx.y;
  const int pend = shared ? min(nprob, pbeg + XS_PCACHE) : blockIdx.y + 1;
  bool any = false;
  for (int p = pbeg; p < pend; ++p) any = any || !prm[p].done;
  if (!any) return;
  load_tw_x<T, N2>(tw, twg);
  // parameters of the block's problems in T, converted once per block:
  // (g_c, B0_c) for c = 0..2, then A0, eta, Pe, Fc
  __shared__ T spar[XS_PCACHE][10];
  for (int i = threadIdx.x; pbeg + i < pend; i += blockDim.x) {
    const SoluteDev& Q = prm[pbeg + i];
    for (int c = 0; c < 3; ++c) {
      spar[i][2 * c] = (T)Q.g[c];
      spar[i][2 * c + 1] = (T)Q.B0[c];
    }
    spar[i][6] = (T)Q.A0;
    spar[i][7] = (T)Q.eta;
    spar[i][8] = (T)Q.Pe;
    spar[i][9] = (T)Q.Fc;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ll = lane / TL, t = lane % TL;
  const unsigned mask = xl_mask();
  cx<T>* b0 = lines + (warp * LPW + ll) * LB;
  cx<T>* b1 = b0 + LS;
  const int ngroups = g.n0 * g.n1 / LPW;
  const int gbase = (blockIdx.x * XS_WARPS + warp) * gpw;
#pragma unroll 1
  for (int gi = 0; gi < gpw; ++gi) {
    const int grp = gbase + gi;
    if (grp >= ngroups) break;
    const long long line = (long long)grp * LPW + ll;
    const long long v0 = line * N2;
    // the indicator is the same for every problem of the loop (hs = 0 when shared)
    const long long hcell = (long long)(pbeg / g.lph) * g.hs;
    const unsigned hm = xl_hmask<N2, TL, E>(Hb + hcell / 32, H + hcell, line, t);
#pragma unroll 1
    for (int p = pbeg; p < pend; ++p) {
      const SoluteDev* P = prm + p;
      if (P->done) continue;
      cx<T>* sp = spec + (long long)p * 4 * g.S;
      const T* up = u + (long long)p * g.us;
      const cx<T>* srow = sp + line * g.P;
      // spectrum rows of d0 chi and d1 chi (that of chi follows into b0 later)
      __syncwarp(mask);
      for (int e = t; e <= M; e += TL) {
        cp_async<(int)sizeof(cx<T>)>(&b0[pad(e)], &srow[e]);
        cp_async<(int)sizeof(cx<T>)>(&b1[pad(e)], &srow[g.S + e]);
      }
      cp_async_commit();
#pragma unroll
      for (int m = 0; m < E; ++m) {
        T2 z;
        z.x = (T)0;
        z.y = (T)0;
        acc[m * 32 + lane] = z;
      }
      cp_async_wait<0>();
      __syncwarp(mask);
      cx<T> v[E];
      // components 0..2: tau_c from the gradient of chi; component 3: s
#pragma unroll 1
      for (int c = 0; c < 4; ++c) {
        cx<T>* bc = c == 1 ? b1 : b0;
        if (c < 3) {
          xl_inverse<T, N2>(bc, tw, t, mask, v);
          const T* q = spar[p - pbeg];
          const T gc = q[2 * c], Bc = q[2 * c + 1], A0 = q[6], eta = q[7], Pe = q[8];
          const T* uc = up + c * g.V + v0;
#pragma unroll
          for (int m = 0; m < E; ++m) {
            const int k = t + TL * m;
            const bool sa = (hm >> (2 * m)) & 1u, sb = (hm >> (2 * m + 1)) & 1u;
            T2 uu;
            if (sa && sb) {
              uu.x = (T)0;
              uu.y = (T)0;
            } else {
              uu = *reinterpret_cast<const T2*>(uc + 2 * k);
            }
            const T ea = v[m].x + gc, eb = v[m].y + gc;
            T2 a2 = acc[m * 32 + lane];
            a2.x += (Bc - (sa ? (T)0 : Pe * uu.x)) * ea;
            a2.y += (Bc - (sb ? (T)0 : Pe * uu.y)) * eb;
            acc[m * 32 + lane] = a2;
            v[m].x = ((sa ? eta : (T)1) - A0) * ea;
            v[m].y = ((sb ? eta : (T)1) - A0) * eb;
          }
          if (CEN && c == 2) {
            // s += D2 tau_2: the neighbours of the lane's pair 2k, 2k+1 are
            // voxel 2k - 1 (lane t - 1, or lane TL - 1 at position m - 1) and
            // 2k + 2 (lane t + 1, or lane 0 at position m + 1); each lane hands
            // on the value its neighbour needs
            const T hc = (T)(N2 / 2);
            const int lb = lane - t;
            const int src_r = lb + (t + 1) % TL, src_l = lb + (t + TL - 1) % TL;
#pragma unroll
            for (int m = 0; m < E; ++m) {
              const T pr = t == 0 ? v[(m + 1) % E].x : v[m].x;
              const T pl = t == TL - 1 ? v[(m + E - 1) % E].y : v[m].y;
              const T right = __shfl_sync(mask, pr, src_r), left = __shfl_sync(mask, pl, src_l);
              T2 a2 = acc[m * 32 + lane];
              a2.x += (v[m].y - left) * hc;
              a2.y += (right - v[m].x) * hc;
              acc[m * 32 + lane] = a2;
            }
            continue;  // tau_2 itself is not transformed
          }
        } else {
          // s = F - (B - B0).(grad chi + g): the accumulated terms plus Pe ubar.g on pore voxels
          // (with CEN also + D2 tau_2)
          const T Fc = spar[p - pbeg][9];
#pragma unroll
          for (int m = 0; m < E; ++m) {
            const bool sa = (hm >> (2 * m)) & 1u, sb = (hm >> (2 * m + 1)) & 1u;
            const T2 a2 = acc[m * 32 + lane];
            v[m] = mk<T>(a2.x + (sa ? (T)0 : Fc), a2.y + (sb ? (T)0 : Fc));
          }
        }
        cx<T> xn;
        xl_forward<T, N2>(bc, tw, t, mask, v, v, xn);
        if (c < 2) {
          cx<T>* dst = sp + c * g.S + line * g.P;
#pragma unroll
          for (int m = 0; m < E; ++m) dst[t + TL * m] = v[m];
          if (t == 0) dst[M] = xn;
          if (c == 0) {
            // the row of chi into b0, hidden behind component 1
            __syncwarp(mask);
            for (int e = t; e <= M; e += TL) cp_async<(int)sizeof(cx<T>)>(&b0[pad(e)], &srow[2 * g.S + e]);
            cp_async_commit();
          } else {
            cp_async_wait<0>();
            __syncwarp(mask);
          }
        } else if (c == 2) {
          // i d2 tau_2^ waits in b1 (own positions only)
#pragma unroll
          for (int m = 0; m < E; ++m) b1[pad(t + TL * m)] = cscale(mul_i(v[m]), d2[t + TL * m]);
          if (t == 0) b1[pad(M)] = cscale(mul_i(xn), d2[M]);
        } else if (CEN) {
          cx<T>* dst = sp + 2 * g.S + line * g.P;
#pragma unroll
          for (int m = 0; m < E; ++m) dst[t + TL * m] = v[m];
          if (t == 0) dst[M] = xn;
        } else {
          cx<T>* dst = sp + 2 * g.S + line * g.P;
#pragma unroll
          for (int m = 0; m < E; ++m) dst[t + TL * m] = v[m] + b1[pad(t + TL * m)];
          if (t == 0) dst[M] = xn + b1[pad(M)];
        }
      }
    }
  }
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

// Line-resident C2R along the contiguous axis (acm_xline.cuh): a warp owns
// LPW lines of one component at a time; the row arrives by cp.async, the
// inverse transform leaves the voxel pairs 2k, 2k+1 (k = t + TL m) of the lane
// in registers, and they are stored as vectors. blockIdx.y = problem * nc +
// component.
template <typename T, int N2>
__global__ void __launch_bounds__(XS_WARPS * 32) k_x_c2r_lr(const cx<T>* __restrict__ spec, T* __restrict__ out,
                                                           Geo g, int nc, long long outProbStride,
                                                           long long specProbStride, const cx<T>* __restrict__ twg) {
  using L = XL<T, N2>;
  constexpr int M = L::M, E = L::E, TL = L::TL, LPW = L::LPW;
  constexpr int LB = L::template lb<1>();
  using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* tw = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* lines = tw + xs_tw_slots<T, N2>();
  const int p = blockIdx.y / nc, c = blockIdx.y % nc;
  load_tw_x<T, N2>(tw, twg);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ll = lane / TL, t = lane % TL;
  const unsigned mask = xl_mask();
  cx<T>* bl = lines + (warp * LPW + ll) * LB;
  const cx<T>* sp = spec + p * specProbStride + c * g.S;
  T* op = out + p * outProbStride + c * g.V;
  const int ngroups = g.n0 * g.n1 / LPW;
  const int gbase = (blockIdx.x * XS_WARPS + warp) * XS_GPW;
#pragma unroll 1
  for (int gi = 0; gi < XS_GPW; ++gi) {
    const int grp = gbase + gi;
    if (grp >= ngroups) break;
    const long long line = (long long)grp * LPW + ll;
    __syncwarp(mask);  // the previous line's readers of bl are done
    for (int e = t; e <= M; e += TL) cp_async<(int)sizeof(cx<T>)>(&bl[pad(e)], &sp[line * g.P + e]);
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp(mask);
    cx<T> v[E];
    xl_inverse<T, N2>(bl, tw, t, mask, v);
    T* orow = op + line * N2;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      T2 w;
      w.x = v[m].x;
      w.y = v[m].y;
      *reinterpret_cast<T2*>(orow + 2 * (t + TL * m)) = w;
    }
  }
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
// OP_INV_SOL (y inverse): (a, b) in, lines (a, i d1 b, i d2 b) inverse-transformed out.
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
  int nouter;       // register-resident passes: pencils along the other strided axis
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

// Transforms the tile's lines (line = component * TX + column); lines of the
// columns w..TX-1 that a tile at the end of a pencil leaves empty are skipped.
template <typename T, int N, int OP, int NC, int TX, int SIGN, int NLINES>
__device__ __forceinline__ void s_fft(cx<T>* sm, const cx<T>* tw, int w) {
  using C = SCfg<T, N, OP, NC, TX>;
  constexpr int per_round = C::NT / C::TL;
#pragma unroll 1
  for (int r = 0; r < C::ROUNDS; ++r) {
    const int job = r * per_round + threadIdx.x / C::TL;
    const bool live = job < NLINES && job % TX < w;
    const unsigned mask = __ballot_sync(0xffffffffu, live);
    if (live) fft_line<T, N, SIGN>(sm + job * C::LS, threadIdx.x % C::TL, tw, mask);
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
  __shared__ T red[4 * 32];
  // the operator's parameters, converted once per block: (nu, beta, b) or
  // (A0, B0), and 1/V
  __shared__ T opar[5];
  const int p = blockIdx.z, outer = blockIdx.y, kx0 = blockIdx.x * TX;
  if (a.sprm && a.sprm[p].done) return;
  if (a.cprm && a.cprm[p].done) return;
  if constexpr (OP == OP_STOKES) {
    if (threadIdx.x == 0) {
      opar[0] = (T)a.sprm[p].nu;
      opar[1] = (T)a.sprm[p].psi[1];
      opar[2] = (T)a.sprm[p].psi[2];
      opar[4] = (T)a.invV;
    }
  } else if constexpr (OP == OP_SOLUTE) {
    if (threadIdx.x == 0) {
      opar[0] = (T)a.cprm[p].A0;
      for (int k = 0; k < 3; ++k) opar[1 + k] = (T)a.cprm[p].B0[k];
      opar[4] = (T)a.invV;
    }
  }
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
      // line 1 = i d1(ky) b: the axis-1 derivative of chi before its inverse
      // transform (the axis-2 one, a factor per column, is applied at the store)
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
    s_fft<T, N, OP, NC, TX, +1, NC * TX>(sm, tw, w);
  } else {
    s_fft<T, N, OP, NC, TX, -1, NIN * TX>(sm, tw, w);
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
    s_fft<T, N, OP, NC, TX, +1, NC * TX>(sm, tw, w);
  }
  if constexpr (OP == OP_STOKES || OP == OP_SOLUTE) {
    __syncthreads();
    const T invV = opar[4];
    const int ky = outer;
    const T d1 = a.sym.d1[ky], l1 = a.sym.l1[ky];
    T acc0 = 0, acc1 = 0, acc2 = 0;
    // hoisted parameters of the operator
    T nu = 0, beta = 0, b = 0, A0 = 0, B00 = 0, B01 = 0, B02 = 0;
    if constexpr (OP == OP_STOKES) {
      nu = opar[0];
      beta = opar[1];
      b = opar[2];
    } else {
      A0 = opar[0];
      B00 = opar[1];
      B01 = opar[2];
      B02 = opar[3];
    }
    // The operator state (q^ and div^, or chi^) is read and rewritten in place:
    // each chunk loads its state before any store (see k_x_stokes_local).
    // The block size is a multiple of TX, so a thread keeps one tile column and
    // its kx symbols and Parseval weight stay in registers.
    static_assert(C::NT % TX == 0, "one column per thread");
    constexpr int TOT = N * TX, CH = 4;
    const int col = threadIdx.x % TX, kx = kx0 + col;
    const bool colok = col < w;
    const T d2 = colok ? a.sym.d2[kx] : (T)0, l2 = colok ? a.sym.l2[kx] : (T)0;
    const T wgt = (kx == 0 || kx == a.nkx) ? (T)1 : (T)2;
    const T l12 = l1 + l2, d12 = d1 * d1 + d2 * d2;
    const long long gcol = (long long)p * a.compStride + (long long)outer * a.outerStride + kx0 + col;
#pragma unroll 1
    for (int base = 0; base < TOT; base += CH * C::NT) {
      bool ok[CH];
      long long gis[CH];
      cx<T> sa[CH], sb[CH];
#pragma unroll
      for (int k = 0; k < CH; ++k) {
        const int idx = base + k * C::NT + threadIdx.x;
        const int j = idx / TX;
        ok[k] = idx < TOT && colok;
        gis[k] = gcol + (long long)j * a.rowStride;
        sa[k] = ok[k] ? a.st0[gis[k]] : mk<T>(0, 0);
        if constexpr (OP == OP_STOKES) sb[k] = ok[k] ? a.st1[gis[k]] : mk<T>(0, 0);
      }
#pragma unroll
      for (int k = 0; k < CH; ++k) {
        if (!ok[k]) continue;
        const int idx = base + k * C::NT + threadIdx.x;
        const int j = idx / TX;
        const long long gi = gis[k];
        const T d0 = a.sym.d0[j], l0 = a.sym.l0[j];
        const T L = l0 + l12, dd = d0 * d0 + d12;
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
    T v3[3] = {acc0, acc1, acc2};
    const int nb = gridDim.x * gridDim.y;
    block_sum_store<3>(v3, red, a.part + ((long long)p * nb + blockIdx.y * gridDim.x + blockIdx.x) * 4);
    __syncthreads();
    s_fft<T, N, OP, NC, TX, +1, NOUT * TX>(sm, tw, w);
  }
  __syncthreads();
  // OP_INV_SOL: line 2 leaves as i d2(kx) b; with NT a multiple of TX every
  // thread stores one column, whose symbol is read once
  constexpr bool fixed_col = C::NT % TX == 0;
  T d2c = (T)0;
  if constexpr (OP == OP_INV_SOL && fixed_col)
    if ((int)threadIdx.x % TX < w) d2c = a.sym.d2[kx0 + (int)threadIdx.x % TX];
  for (int idx = threadIdx.x; idx < NOUT * N * TX; idx += blockDim.x) {
    const int col = idx % TX, j = (idx / TX) % N, c = idx / (TX * N);
    if (col < w) {
      cx<T> x = sm[(c * TX + col) * C::LS + pad(j)];
      if constexpr (OP == OP_INV_SOL)
        if (c == 2) x = cscale(mul_i(x), fixed_col ? d2c : a.sym.d2[kx0 + col]);
      base[c * a.compStride + j * a.rowStride + col] = x;
    }
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
    // predicated (not early-exit) iterations, so the loads of an unrolled
    // group are all in flight together
#pragma unroll 4
    for (int k = 0; k < CHK; ++k) {
      const long long v = v0 + k * stride;
      const bool in = v < V;
      const T a = in ? up[v] : (T)0, b = in ? up[V + v] : (T)0, cc = in ? up[2 * V + v] : (T)0;
      const bool pore = in && Hp[in ? v : 0] == 0;
      c[0] += a;
      c[1] += b;
      c[2] += cc;
      c[3] += pore ? a : (T)0;
      c[4] += pore ? b : (T)0;
      c[5] += pore ? cc : (T)0;
      c[6] += pore ? (T)1 : (T)0;
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
    // predicated (not early-exit) iterations, so the loads of an unrolled
    // group are all in flight together
#pragma unroll 4
    for (int k = 0; k < CHK; ++k) {
      const long long v = v0 + k * stride;
      const bool in = v < V;
      const long long vi = in ? v : 0;
      const T ch = cp[vi];
      const bool pore = Hp[vi] == 0;
      const T A = pore ? (T)1 : eta;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const T gi = gg[i] + gp[i * V + vi];
        const T pe = pore ? Pe * (ub[i] - up[i * V + vi]) * ch : (T)0;
        c[i] += (in && pore) ? gi + pe : (T)0;
        c[3 + i] += in ? A * gi + pe : (T)0;
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
    // predicated (not early-exit) iterations, so the loads of an unrolled
    // group are all in flight together
#pragma unroll 4
    for (int k = 0; k < CHK; ++k) {
      const long long v = v0 + k * stride;
      const long long vi = v < V ? v : 0;
      const bool use = v < V && H[vi] == 0;
      const T a = use ? f[vi] : (T)0, b = use ? f[V + vi] : (T)0, d = use ? f[2 * V + vi] : (T)0;
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

#include "acm_rpass.cuh"
