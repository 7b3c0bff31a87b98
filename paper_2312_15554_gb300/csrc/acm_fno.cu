// acm_fno.cu -- the learned warm start: a 3D Fourier neural operator with
// hand-written forward and backward kernels (BF16 weights and stored
// activations, FP32 arithmetic and accumulation) and an AdamW step.
//
// Model (width W, `modes` per axis, L layers) on a grid (n0, n1, n2):
//   features a = (H, x0, x1, x2) with x_c = (i_c + 1/2)/n_c
//   lift     v0 = P a + p
//   layer l  v_{l+1} = gelu(z_l),  z_l = G(R_l F(v_l)) + M_l v_l + m_l
//            F: forward DFT on the kept modes; G(Y) = (1/V) sum_k w_k Re[Y(k) e^{2 pi i k.x/n}]
//            (w_k = 1 on the k2 = 0 plane, 2 elsewhere); R_l(k): W x W complex per kept mode
//   project  out = Q v_L + q   (u and lambda, 6 channels)
// Kept modes: k2 in [0, modes), k1 and k0 in [0, modes) U [n - modes, n).
// Loss: (1/(B V)) sum [ |out_u - t_u|^2 + H |out_lambda - t_lambda|^2 ].
// F and G run on the library's FFT passes; the per-mode channel mix, the
// pointwise layers, the projection and the weight gradients are kernels here.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "acm.h"
#include "acm_fft.cuh"
#include "acm_ops.h"

using namespace acm;

namespace {

constexpr int NRB = 512;  // blocks (partials) of the weight-gradient reductions

struct FnoDims {
  int n0, n1, n2, W, md, L;
  long long V;
  int M;  // kept modes
};

__host__ __device__ inline int mode_index_axis(int j, int md, int n) { return j < md ? j : n - 2 * md + j; }

__device__ __forceinline__ float bf(const __nv_bfloat16 x) { return __bfloat162float(x); }

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.3989422804014327f * expf(-0.5f * z * z);
}

// ---------------------------------------------------------------------------
// lift: v0[b][c][x] = sum_a P[c][a] a_a(x) + p[c]
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(256) k_lift(const uint8_t* __restrict__ H, const __nv_bfloat16* __restrict__ P,
                                             const __nv_bfloat16* __restrict__ pb, __nv_bfloat16* __restrict__ v0,
                                             FnoDims d, int B) {
  __shared__ float sP[W * 4], sp[W];
  for (int i = threadIdx.x; i < W * 4; i += blockDim.x) sP[i] = bf(P[i]);
  for (int i = threadIdx.x; i < W; i += blockDim.x) sp[i] = bf(pb[i]);
  __syncthreads();
  const long long total = (long long)B * d.V;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / d.V, x = t - b * d.V;
    const int i2 = (int)(x % d.n2), i1 = (int)((x / d.n2) % d.n1), i0 = (int)(x / ((long long)d.n2 * d.n1));
    const float a[4] = {(float)H[t], (i0 + 0.5f) / d.n0, (i1 + 0.5f) / d.n1, (i2 + 0.5f) / d.n2};
    __nv_bfloat16* o = v0 + b * W * d.V + x;
#pragma unroll 4
    for (int c = 0; c < W; ++c)
      o[c * d.V] = __float2bfloat16(sp[c] + sP[c * 4] * a[0] + sP[c * 4 + 1] * a[1] + sP[c * 4 + 2] * a[2] +
                                    sP[c * 4 + 3] * a[3]);
  }
}

__global__ void k_bf16_to_f32(const __nv_bfloat16* __restrict__ in, float* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = bf(in[i]);
}

// kept modes of C fields [C][S] (half spectrum, pitch P) -> X[C][M], times scale[w_k]
__global__ void k_gather(const cx<float>* __restrict__ spec, cx<float>* __restrict__ X, FnoDims d, Geo g, int C,
                         float s0, float s1) {
  const long long total = (long long)C * d.M;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / d.M), m = (int)(t - (long long)c * d.M);
    const int j2 = m % d.md, j1 = (m / d.md) % (2 * d.md), j0 = m / (2 * d.md * d.md);
    const int i0 = mode_index_axis(j0, d.md, d.n0), i1 = mode_index_axis(j1, d.md, d.n1);
    const cx<float> v = spec[c * g.S + ((long long)i0 * d.n1 + i1) * g.P + j2];
    const float s = j2 == 0 ? s0 : s1;
    X[t] = mk<float>(v.x * s, v.y * s);
  }
}

// X[C][M] (times scale[w_k]) -> kept modes of a zeroed half spectrum
__global__ void k_scatter(const cx<float>* __restrict__ X, cx<float>* __restrict__ spec, FnoDims d, Geo g, int C,
                          float s0, float s1) {
  const long long total = (long long)C * d.M;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / d.M), m = (int)(t - (long long)c * d.M);
    const int j2 = m % d.md, j1 = (m / d.md) % (2 * d.md), j0 = m / (2 * d.md * d.md);
    const int i0 = mode_index_axis(j0, d.md, d.n0), i1 = mode_index_axis(j1, d.md, d.n1);
    const float s = j2 == 0 ? s0 : s1;
    const cx<float> v = X[t];
    spec[c * g.S + ((long long)i0 * d.n1 + i1) * g.P + j2] = mk<float>(v.x * s, v.y * s);
  }
}

// real-part semantics of G on the k2 = 0 column: drop the imaginary part of
// column 0 after the transforms along axes 0 and 1
__global__ void k_real_col0(cx<float>* __restrict__ spec, Geo g, int C) {
  const long long rows = (long long)g.n0 * g.n1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)C * rows;
       t += (long long)gridDim.x * blockDim.x) {
    const long long c = t / rows, r = t - c * rows;
    spec[c * g.S + r * g.P].y = 0.0f;
  }
}

// per mode: Y[b][i] = sum_j R[i][j] X[b][j]
template <int W>
__global__ void __launch_bounds__(256) k_mix_fwd(const cx<float>* __restrict__ X, const __nv_bfloat16* __restrict__ R,
                                                cx<float>* __restrict__ Y, FnoDims d, int B) {
  __shared__ cx<float> sR[W * W];
  __shared__ cx<float> sX[64 * W];
  const int m = blockIdx.x;
  const __nv_bfloat16* Rm = R + (long long)m * W * W * 2;
  for (int e = threadIdx.x; e < W * W; e += blockDim.x) sR[e] = mk<float>(bf(Rm[2 * e]), bf(Rm[2 * e + 1]));
  for (int e = threadIdx.x; e < B * W; e += blockDim.x) sX[e] = X[(long long)e * d.M + m];
  __syncthreads();
  for (int e = threadIdx.x; e < B * W; e += blockDim.x) {
    const int b = e / W, i = e - b * W;
    cx<float> acc = mk<float>(0.f, 0.f);
#pragma unroll 8
    for (int j = 0; j < W; ++j) acc = acc + cmul(sR[i * W + j], sX[b * W + j]);
    Y[(long long)e * d.M + m] = acc;
  }
}

// per mode: gR[i][j] = sum_b gY[b][i] conj(X[b][j]);  gX[b][j] = sum_i conj(R[i][j]) gY[b][i]
template <int W>
__global__ void __launch_bounds__(256) k_mix_bwd(const cx<float>* __restrict__ X, const cx<float>* __restrict__ gY,
                                                const __nv_bfloat16* __restrict__ R, float* __restrict__ gR,
                                                cx<float>* __restrict__ gX, FnoDims d, int B) {
  __shared__ cx<float> sR[W * W];
  __shared__ cx<float> sX[64 * W], sG[64 * W];
  const int m = blockIdx.x;
  const __nv_bfloat16* Rm = R + (long long)m * W * W * 2;
  for (int e = threadIdx.x; e < W * W; e += blockDim.x) sR[e] = mk<float>(bf(Rm[2 * e]), bf(Rm[2 * e + 1]));
  for (int e = threadIdx.x; e < B * W; e += blockDim.x) {
    sX[e] = X[(long long)e * d.M + m];
    sG[e] = gY[(long long)e * d.M + m];
  }
  __syncthreads();
  float* gRm = gR + (long long)m * W * W * 2;
  for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
    const int i = e / W, j = e - i * W;
    cx<float> acc = mk<float>(0.f, 0.f);
    for (int b = 0; b < B; ++b) acc = acc + cmul(sG[b * W + i], cconj(sX[b * W + j]));
    gRm[2 * e] = acc.x;
    gRm[2 * e + 1] = acc.y;
  }
  for (int e = threadIdx.x; e < B * W; e += blockDim.x) {
    const int b = e / W, j = e - b * W;
    cx<float> acc = mk<float>(0.f, 0.f);
#pragma unroll 8
    for (int i = 0; i < W; ++i) acc = acc + cmul(cconj(sR[i * W + j]), sG[b * W + i]);
    gX[(long long)e * d.M + m] = acc;
  }
}

// z = y + M v + m ; v' = gelu(z)   (per voxel)
template <int W>
__global__ void __launch_bounds__(256) k_pointwise_fwd(const float* __restrict__ y, const __nv_bfloat16* __restrict__ v,
                                                      const __nv_bfloat16* __restrict__ Mw,
                                                      const __nv_bfloat16* __restrict__ mb,
                                                      __nv_bfloat16* __restrict__ z, __nv_bfloat16* __restrict__ vout,
                                                      FnoDims d, int B) {
  __shared__ float sM[W * W], sm[W];
  for (int i = threadIdx.x; i < W * W; i += blockDim.x) sM[i] = bf(Mw[i]);
  for (int i = threadIdx.x; i < W; i += blockDim.x) sm[i] = bf(mb[i]);
  __syncthreads();
  const long long total = (long long)B * d.V;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / d.V, x = t - b * d.V;
    const long long base = b * W * d.V + x;
    float vv[W];
#pragma unroll
    for (int j = 0; j < W; ++j) vv[j] = bf(v[base + j * d.V]);
#pragma unroll 4
    for (int i = 0; i < W; ++i) {
      float acc = y[base + i * d.V] + sm[i];
#pragma unroll
      for (int j = 0; j < W; ++j) acc += sM[i * W + j] * vv[j];
      z[base + i * d.V] = __float2bfloat16(acc);
      vout[base + i * d.V] = __float2bfloat16(gelu_f(acc));
    }
  }
}

// dz = dv * gelu'(z) ; dvM = M^T dz   (per voxel)
template <int W>
__global__ void __launch_bounds__(256) k_act_bwd(const float* __restrict__ dv, const __nv_bfloat16* __restrict__ z,
                                                const __nv_bfloat16* __restrict__ Mw, float* __restrict__ dz,
                                                float* __restrict__ dvM, FnoDims d, int B) {
  __shared__ float sM[W * W];
  for (int i = threadIdx.x; i < W * W; i += blockDim.x) sM[i] = bf(Mw[i]);
  __syncthreads();
  const long long total = (long long)B * d.V;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / d.V, x = t - b * d.V;
    const long long base = b * W * d.V + x;
    float g[W];
#pragma unroll
    for (int i = 0; i < W; ++i) {
      g[i] = dv[base + i * d.V] * gelu_grad_f(bf(z[base + i * d.V]));
      dz[base + i * d.V] = g[i];
    }
#pragma unroll 4
    for (int j = 0; j < W; ++j) {
      float acc = 0.f;
#pragma unroll
      for (int i = 0; i < W; ++i) acc += sM[i * W + j] * g[i];
      dvM[base + j * d.V] = acc;
    }
  }
}

__global__ void k_add(float* __restrict__ a, const float* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    a[i] += b[i];
}

// projection, loss and its gradient: out = Q v + q; d = (out - t) * mask;
// dout = 2 d / (B V); partial sums of d^2 per block
template <int W>
__global__ void __launch_bounds__(256) k_project(const __nv_bfloat16* __restrict__ v, const __nv_bfloat16* __restrict__ Q,
                                                const __nv_bfloat16* __restrict__ q, const float* __restrict__ target,
                                                const uint8_t* __restrict__ H, float* __restrict__ out,
                                                float* __restrict__ dout, double* __restrict__ lpart, FnoDims d, int B) {
  __shared__ float sQ[6 * W], sq[6];
  __shared__ double red[32];
  for (int i = threadIdx.x; i < 6 * W; i += blockDim.x) sQ[i] = bf(Q[i]);
  for (int i = threadIdx.x; i < 6; i += blockDim.x) sq[i] = bf(q[i]);
  __syncthreads();
  const long long total = (long long)B * d.V;
  const float sc = 2.0f / (float)total;
  float acc = 0.f;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / d.V, x = t - b * d.V;
    float r6[6];
#pragma unroll
    for (int o = 0; o < 6; ++o) r6[o] = sq[o];
#pragma unroll 4
    for (int j = 0; j < W; ++j) {
      const float vj = bf(v[b * W * d.V + j * d.V + x]);
#pragma unroll
      for (int o = 0; o < 6; ++o) r6[o] += sQ[o * W + j] * vj;
    }
    const bool solid = H[t] != 0;
#pragma unroll
    for (int o = 0; o < 6; ++o) {
      const float r = r6[o];
      const long long oi = (b * 6 + o) * d.V + x;
      if (out) out[oi] = r;
      if (target) {
        const float dd = (o < 3 || solid) ? r - target[oi] : 0.f;
        acc += dd * dd;
        dout[oi] = sc * dd;
      }
    }
  }
  if (!target) return;
  double a = acc;
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    lpart[blockIdx.x] = s;
  }
}

// dv = Q^T dout
template <int W>
__global__ void __launch_bounds__(256) k_project_bwd(const float* __restrict__ dout, const __nv_bfloat16* __restrict__ Q,
                                                    float* __restrict__ dv, FnoDims d, int B) {
  __shared__ float sQ[6 * W];
  for (int i = threadIdx.x; i < 6 * W; i += blockDim.x) sQ[i] = bf(Q[i]);
  __syncthreads();
  const long long total = (long long)B * d.V;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / d.V, x = t - b * d.V;
    float g[6];
#pragma unroll
    for (int o = 0; o < 6; ++o) g[o] = dout[(b * 6 + o) * d.V + x];
#pragma unroll 4
    for (int j = 0; j < W; ++j) {
      float acc = 0.f;
#pragma unroll
      for (int o = 0; o < 6; ++o) acc += sQ[o * W + j] * g[o];
      dv[b * W * d.V + j * d.V + x] = acc;
    }
  }
}

// Weight gradients G[i][j] = sum_x A_i(x) Bj(x) and g[i] = sum_x A_i(x) over all
// voxels of the batch, as NRB block partials [NRB][AD * BD + AD].
// A: FP32 [b][AD][V]. B: BF16 [b][BD][V], or the features (H, x0, x1, x2) when LIFT.
template <int AD, int BD, bool LIFT>
__global__ void __launch_bounds__(256) k_wgrad(const float* __restrict__ A, const __nv_bfloat16* __restrict__ Bv,
                                              const uint8_t* __restrict__ H, float* __restrict__ part, FnoDims d,
                                              int B) {
  constexpr int TV = 64;
  constexpr int NE = AD * BD + AD;
  __shared__ float sA[AD][TV], sB[BD][TV];
  float acc[(NE + 255) / 256];
#pragma unroll
  for (int k = 0; k < (NE + 255) / 256; ++k) acc[k] = 0.f;
  const long long total = (long long)B * d.V;
  const long long per = (total + gridDim.x - 1) / gridDim.x;
  const long long lo = blockIdx.x * per, hi = min(total, lo + per);
  for (long long t0 = lo; t0 < hi; t0 += TV) {
    for (int e = threadIdx.x; e < (AD + BD) * TV; e += blockDim.x) {
      const int c = e / TV, k = e - c * TV;
      const long long t = t0 + k;
      float val = 0.f;
      if (t < hi) {
        const long long b = t / d.V, x = t - b * d.V;
        if (c < AD) {
          val = A[(b * AD + c) * d.V + x];
        } else {
          const int cb = c - AD;
          if constexpr (LIFT) {
            if (cb == 0) val = (float)H[t];
            else {
              const int i2 = (int)(x % d.n2), i1 = (int)((x / d.n2) % d.n1), i0 = (int)(x / ((long long)d.n2 * d.n1));
              val = cb == 1 ? (i0 + 0.5f) / d.n0 : (cb == 2 ? (i1 + 0.5f) / d.n1 : (i2 + 0.5f) / d.n2);
            }
          } else {
            val = bf(Bv[(b * BD + cb) * d.V + x]);
          }
        }
      }
      if (c < AD) sA[c][k] = val;
      else sB[c - AD][k] = val;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < (NE + 255) / 256; ++k) {
      const int e = threadIdx.x + 256 * k;
      if (e < AD * BD) {
        const int i = e / BD, j = e - i * BD;
        float s = 0.f;
#pragma unroll 8
        for (int v = 0; v < TV; ++v) s += sA[i][v] * sB[j][v];
        acc[k] += s;
      } else if (e < NE) {
        const int i = e - AD * BD;
        float s = 0.f;
#pragma unroll 8
        for (int v = 0; v < TV; ++v) s += sA[i][v];
        acc[k] += s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < (NE + 255) / 256; ++k) {
    const int e = threadIdx.x + 256 * k;
    if (e < NE) part[(long long)blockIdx.x * NE + e] = acc[k];
  }
}

// sum the NRB partials: out_w[e] for e < AD*BD, out_b[e] for the biases
__global__ void k_reduce_parts(const float* __restrict__ part, int ne, int nab, float* __restrict__ out_w,
                               float* __restrict__ out_b) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
    double s = 0;
    for (int r = 0; r < NRB; ++r) s += part[(long long)r * ne + e];
    if (e < nab) out_w[e] = (float)s;
    else out_b[e - nab] = (float)s;
  }
}

__global__ void k_adamw(float* __restrict__ th, __nv_bfloat16* __restrict__ tb, const float* __restrict__ g,
                        float* __restrict__ m1, float* __restrict__ m2, long long n, float lr, float b1, float b2,
                        float eps, float wd, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    const float t = th[i] - lr * ((a / c1) / (sqrtf(v / c2) + eps) + wd * th[i]);
    th[i] = t;
    tb[i] = __float2bfloat16(t);
  }
}

__global__ void k_f32_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16(in[i]);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct acm_fno {
  FnoDims d;
  Geo g;
  int Bmax;
  cudaStream_t st;
  long long np;
  // parameter offsets (elements) in the flat vector
  long long oP, op, oQ, oq;
  std::vector<long long> oR, oM, om;
  float* theta = nullptr;          // FP32 master
  __nv_bfloat16* tb = nullptr;     // BF16 copy used by the kernels
  float* grad = nullptr;
  float* m1 = nullptr;
  float* m2 = nullptr;
  long long step = 0;
  // activations
  __nv_bfloat16* v = nullptr;      // [L+1][Bmax][W][V]
  __nv_bfloat16* z = nullptr;      // [L][Bmax][W][V]
  cx<float>* X = nullptr;          // [L][Bmax][W][M]
  cx<float>* Y = nullptr;          // [Bmax][W][M]
  float* r0 = nullptr;             // [Bmax][W][V] FP32 scratch
  float* r1 = nullptr;             // [Bmax][W][V] FP32 scratch
  float* r2 = nullptr;             // [Bmax][W][V] FP32 scratch
  float* dout = nullptr;           // [Bmax][6][V]
  float* tgt = nullptr;            // [Bmax][6][V] staging of host targets
  uint8_t* Hs = nullptr;           // [Bmax][V] staging of indicators
  uint8_t* Hp = nullptr;           // [Bmax][V] axis-swapped indicators (warm start, allocated on first use)
  cx<float>* spec = nullptr;       // [Bmax * W][S]
  float* part = nullptr;           // [NRB][W*W + W]
  double* lpart = nullptr;         // [NRB]
  void* tw = nullptr;              // FP32 twiddles
};

namespace {

#define FK(x)                              \
  do {                                     \
    if ((x) != cudaSuccess) {              \
      cudaGetLastError();                  \
      return ACM_ERR_CUDA;                 \
    }                                      \
  } while (0)

#define CKF(x)                   \
  do {                           \
    acm_status s_ = (x);         \
    if (s_ != ACM_OK) return s_; \
  } while (0)

int blocks_for(long long n) { return (int)std::min<long long>(4 * 152, (n + 255) / 256); }

acm_status fft_fwd(acm_fno* f, const float* in, int C) {
  Sym<float> none = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  FK(Ops<float>::x_r2c(f->g, C, 1, f->spec, f->g.S, in, f->g.V, f->tw, f->st));
  FK(Ops<float>::pass(f->g, 1, P_FWD, 1, C, f->spec, f->g.S, none, f->tw, nullptr, nullptr, nullptr, nullptr, nullptr,
                      f->st));
  FK(Ops<float>::pass(f->g, 0, P_FWD, 1, C, f->spec, f->g.S, none, f->tw, nullptr, nullptr, nullptr, nullptr, nullptr,
                      f->st));
  return ACM_OK;
}

// inverse of the kept-mode spectrum with real-part semantics on the k2 = 0 column
acm_status fft_inv(acm_fno* f, float* out, int C, bool scale) {
  Sym<float> none = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  FK(Ops<float>::pass(f->g, 0, scale ? P_INV_SCALE : P_INV, 1, C, f->spec, f->g.S, none, f->tw, nullptr, nullptr,
                      nullptr, nullptr, nullptr, f->st));
  FK(Ops<float>::pass(f->g, 1, P_INV, 1, C, f->spec, f->g.S, none, f->tw, nullptr, nullptr, nullptr, nullptr, nullptr,
                      f->st));
  k_real_col0<<<blocks_for((long long)C * f->g.n0 * f->g.n1), 256, 0, f->st>>>(f->spec, f->g, C);
  FK(cudaGetLastError());
  FK(Ops<float>::x_c2r(f->g, C, 1, f->spec, f->g.S, out, f->g.V, f->tw, f->st));
  return ACM_OK;
}

template <int W>
acm_status fno_forward_impl(acm_fno* f, int B, const uint8_t* Hd, const float* target, float* out, double* loss) {
  const FnoDims& d = f->d;
  const long long BV = (long long)B * d.V;
  const long long act = (long long)f->Bmax * W * d.V;
  const int C = B * W;
  const int nb = blocks_for(BV);
  k_lift<W><<<nb, 256, 0, f->st>>>(Hd, f->tb + f->oP, f->tb + f->op, f->v, d, B);
  FK(cudaGetLastError());
  for (int l = 0; l < d.L; ++l) {
    __nv_bfloat16* vl = f->v + l * act;
    k_bf16_to_f32<<<blocks_for(BV * W), 256, 0, f->st>>>(vl, f->r0, BV * W);
    FK(cudaGetLastError());
    CKF(fft_fwd(f, f->r0, C));
    cx<float>* Xl = f->X + (long long)l * f->Bmax * W * d.M;
    k_gather<<<blocks_for((long long)C * d.M), 256, 0, f->st>>>(f->spec, Xl, d, f->g, C, 1.f, 1.f);
    FK(cudaGetLastError());
    k_mix_fwd<W><<<d.M, 256, 0, f->st>>>(Xl, f->tb + f->oR[l], f->Y, d, B);
    FK(cudaGetLastError());
    FK(cudaMemsetAsync(f->spec, 0, (size_t)C * f->g.S * sizeof(cx<float>), f->st));
    k_scatter<<<blocks_for((long long)C * d.M), 256, 0, f->st>>>(f->Y, f->spec, d, f->g, C, 1.f, 1.f);
    FK(cudaGetLastError());
    CKF(fft_inv(f, f->r1, C, true));
    k_pointwise_fwd<W><<<nb, 256, 0, f->st>>>(f->r1, vl, f->tb + f->oM[l], f->tb + f->om[l], f->z + l * act,
                                              f->v + (l + 1) * act, d, B);
    FK(cudaGetLastError());
  }
  k_project<W><<<NRB, 256, 0, f->st>>>(f->v + d.L * act, f->tb + f->oQ, f->tb + f->oq, target, Hd, out, f->dout,
                                       f->lpart, d, B);
  FK(cudaGetLastError());
  if (loss) {
    std::vector<double> lp(NRB);
    FK(cudaMemcpyAsync(lp.data(), f->lpart, NRB * sizeof(double), cudaMemcpyDeviceToHost, f->st));
    FK(cudaStreamSynchronize(f->st));
    double s = 0;
    for (double x : lp) s += x;
    *loss = s / (double)BV;
  }
  return ACM_OK;
}

template <int AD, int BD, bool LIFT>
acm_status wgrad(acm_fno* f, int B, const float* A, const __nv_bfloat16* Bv, const uint8_t* H, float* gw, float* gb) {
  k_wgrad<AD, BD, LIFT><<<NRB, 256, 0, f->st>>>(A, Bv, H, f->part, f->d, B);
  FK(cudaGetLastError());
  const int ne = AD * BD + AD;
  k_reduce_parts<<<(ne + 255) / 256, 256, 0, f->st>>>(f->part, ne, AD * BD, gw, gb);
  FK(cudaGetLastError());
  return ACM_OK;
}

template <int W>
acm_status fno_backward_impl(acm_fno* f, int B, const uint8_t* Hd) {
  const FnoDims& d = f->d;
  const long long BV = (long long)B * d.V;
  const long long act = (long long)f->Bmax * W * d.V;
  const int C = B * W;
  const int nb = blocks_for(BV);
  const float invV = 1.0f / (float)d.V;
  // projection
  CKF((wgrad<6, W, false>(f, B, f->dout, f->v + d.L * act, nullptr, f->grad + f->oQ, f->grad + f->oq)));
  k_project_bwd<W><<<nb, 256, 0, f->st>>>(f->dout, f->tb + f->oQ, f->r0, d, B);  // r0 = dv
  FK(cudaGetLastError());
  for (int l = d.L - 1; l >= 0; --l) {
    __nv_bfloat16* vl = f->v + l * act;
    // r1 = dz, r2 = M^T dz
    k_act_bwd<W><<<nb, 256, 0, f->st>>>(f->r0, f->z + l * act, f->tb + f->oM[l], f->r1, f->r2, d, B);
    FK(cudaGetLastError());
    CKF((wgrad<W, W, false>(f, B, f->r1, vl, nullptr, f->grad + f->oM[l], f->grad + f->om[l])));
    // gY = (w_k / V) F(dz) on the kept modes
    CKF(fft_fwd(f, f->r1, C));
    k_gather<<<blocks_for((long long)C * d.M), 256, 0, f->st>>>(f->spec, f->Y, d, f->g, C, invV, 2.f * invV);
    FK(cudaGetLastError());
    cx<float>* Xl = f->X + (long long)l * f->Bmax * W * d.M;
    cx<float>* gX = reinterpret_cast<cx<float>*>(f->r1);  // dz no longer needed: reuse as gX [C][M]
    k_mix_bwd<W><<<d.M, 256, 0, f->st>>>(Xl, f->Y, f->tb + f->oR[l], f->grad + f->oR[l], gX, d, B);
    FK(cudaGetLastError());
    // dv(spectral) = sum_k Re[gX e^{i k.x}] = unnormalised inverse of gX / w_k
    FK(cudaMemsetAsync(f->spec, 0, (size_t)C * f->g.S * sizeof(cx<float>), f->st));
    k_scatter<<<blocks_for((long long)C * d.M), 256, 0, f->st>>>(gX, f->spec, d, f->g, C, 1.f, 0.5f);
    FK(cudaGetLastError());
    CKF(fft_inv(f, f->r1, C, false));
    k_add<<<blocks_for(BV * W), 256, 0, f->st>>>(f->r2, f->r1, BV * W);
    FK(cudaGetLastError());
    std::swap(f->r0, f->r2);  // r0 = dv of layer l's input
  }
  CKF((wgrad<W, 4, true>(f, B, f->r0, nullptr, Hd, f->grad + f->oP, f->grad + f->op)));
  return ACM_OK;
}

// Linear index of the voxel whose axes 0 and j (1 or 2) are swapped, on an
// n x n x n grid. The swap is its own inverse.
__device__ __forceinline__ long long swap_axes(long long i, int n, int j) {
  const int c = (int)(i % n), b = (int)((i / n) % n), a = (int)(i / ((long long)n * n));
  return j == 1 ? ((long long)b * n + a) * n + c : ((long long)c * n + b) * n + a;
}

__global__ void k_swap_h(const uint8_t* __restrict__ H, uint8_t* __restrict__ Hp, int n, int j, long long V,
                         long long total) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / V, i = t - b * V;
    Hp[t] = H[b * V + swap_axes(i, n, j)];
  }
}

// Predictions out' [B][6][V] for the load e_0 on the swapped cell become the
// warm start of load e_j on the cell: u_c(x) = u'_{s(c)}(s x) with s the swap
// of 0 and j (the identity for j = 0); the multiplier transforms alike.
// Outputs [B][3 loads][3][V]; this writes the slot of load j.
__global__ void k_unswap_out(const float* __restrict__ o, float* __restrict__ u, float* __restrict__ lam, int n, int j,
                             long long V, long long total) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / V, i = t - b * V;
    const long long si = j == 0 ? i : swap_axes(i, n, j);
    const float* ob = o + b * 6 * V;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int sc = c == j ? 0 : (c == 0 ? j : c);
      const long long dst = ((b * 3 + j) * 3 + c) * V + i;
      u[dst] = ob[sc * V + si];
      lam[dst] = ob[(3 + sc) * V + si];
    }
  }
}

}  // namespace


namespace {

bool fno_on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename F>
acm_status dispatch_w(int W, F&& fn) {
  switch (W) {
    case 4: return fn(std::integral_constant<int, 4>());
    case 8: return fn(std::integral_constant<int, 8>());
    case 16: return fn(std::integral_constant<int, 16>());
    case 32: return fn(std::integral_constant<int, 32>());
    default: return ACM_ERR_ARG;
  }
}

void fno_free(acm_fno* f) {
  void* ps[] = {f->theta, f->tb, f->grad, f->m1, f->m2, f->v, f->z, f->X, f->Y, f->r0, f->r1, f->r2,
                f->dout, f->tgt, f->Hs, f->Hp, f->spec, f->part, f->lpart, f->tw};
  for (void* p : ps)
    if (p) cudaFree(p);
  cudaGetLastError();
}

}  // namespace

extern "C" {

acm_status acm_fno_create(acm_fno** out, int n0, int n1, int n2, int width, int modes, int layers, int max_batch,
                          void* stream) {
  if (!out) return ACM_ERR_ARG;
  *out = nullptr;
  auto p2 = [](int n) { return n >= 8 && n <= 512 && (n & (n - 1)) == 0; };
  if (!p2(n0) || !p2(n1) || !p2(n2)) return ACM_ERR_UNSUPPORTED_SIZE;
  if (!(width == 4 || width == 8 || width == 16 || width == 32) || modes < 1 || 2 * modes > n0 || 2 * modes > n1 ||
      modes > n2 / 2 || layers < 1 || layers > 16 || max_batch < 1 || max_batch > 64)
    return ACM_ERR_ARG;
  acm_fno* f = new (std::nothrow) acm_fno();
  if (!f) return ACM_ERR_NOMEM;
  FnoDims& d = f->d;
  d.n0 = n0;
  d.n1 = n1;
  d.n2 = n2;
  d.W = width;
  d.md = modes;
  d.L = layers;
  d.V = (long long)n0 * n1 * n2;
  d.M = 4 * modes * modes * modes;
  Geo& g = f->g;
  g.n0 = n0;
  g.n1 = n1;
  g.n2 = n2;
  g.Pu = n2 / 2 + 1;
  g.P = n2 / 2 + 4;
  g.V = d.V;
  g.S = (long long)n0 * n1 * g.P;
  g.hs = 0;
  g.us = 0;
  g.lph = 1;
  f->Bmax = max_batch;
  f->st = (cudaStream_t)stream;
  long long o = 0;
  f->oP = o;
  o += 4LL * width;
  f->op = o;
  o += width;
  for (int l = 0; l < layers; ++l) {
    f->oR.push_back(o);
    o += 2LL * d.M * width * width;
    f->oM.push_back(o);
    o += (long long)width * width;
    f->om.push_back(o);
    o += width;
  }
  f->oQ = o;
  o += 6LL * width;
  f->oq = o;
  o += 6;
  f->np = o;
  const long long act = (long long)max_batch * width * d.V;
  const long long ne = (long long)width * width + width;
  bool ok = cudaMalloc(&f->theta, f->np * 4) == cudaSuccess && cudaMalloc(&f->tb, f->np * 2) == cudaSuccess &&
            cudaMalloc(&f->grad, f->np * 4) == cudaSuccess && cudaMalloc(&f->m1, f->np * 4) == cudaSuccess &&
            cudaMalloc(&f->m2, f->np * 4) == cudaSuccess &&
            cudaMalloc(&f->v, (layers + 1) * act * 2) == cudaSuccess &&
            cudaMalloc(&f->z, layers * act * 2) == cudaSuccess &&
            cudaMalloc(&f->X, (long long)layers * max_batch * width * d.M * sizeof(cx<float>)) == cudaSuccess &&
            cudaMalloc(&f->Y, (long long)max_batch * width * d.M * sizeof(cx<float>)) == cudaSuccess &&
            cudaMalloc(&f->r0, act * 4) == cudaSuccess && cudaMalloc(&f->r1, act * 4) == cudaSuccess &&
            cudaMalloc(&f->r2, act * 4) == cudaSuccess &&
            cudaMalloc(&f->dout, (long long)max_batch * 6 * d.V * 4) == cudaSuccess &&
            cudaMalloc(&f->tgt, (long long)max_batch * 6 * d.V * 4) == cudaSuccess &&
            cudaMalloc(&f->Hs, (long long)max_batch * d.V) == cudaSuccess &&
            cudaMalloc(&f->spec, (long long)max_batch * width * g.S * sizeof(cx<float>)) == cudaSuccess &&
            cudaMalloc(&f->part, NRB * ne * 4) == cudaSuccess &&
            cudaMalloc(&f->lpart, NRB * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&f->tw, 2 * TW_MAX * sizeof(float)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    fno_free(f);
    delete f;
    return ACM_ERR_NOMEM;
  }
  std::vector<float> tw(2 * TW_MAX);
  const double PI = 3.14159265358979323846;
  for (int k = 0; k < TW_MAX; ++k) {
    tw[2 * k] = (float)std::cos(2.0 * PI * k / TW_MAX);
    tw[2 * k + 1] = (float)(-std::sin(2.0 * PI * k / TW_MAX));
  }
  if (cudaMemcpy(f->tw, tw.data(), tw.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(f->theta, 0, f->np * 4) != cudaSuccess || cudaMemset(f->tb, 0, f->np * 2) != cudaSuccess ||
      cudaMemset(f->m1, 0, f->np * 4) != cudaSuccess || cudaMemset(f->m2, 0, f->np * 4) != cudaSuccess ||
      cudaMemset(f->grad, 0, f->np * 4) != cudaSuccess ||
      cudaMemset(f->spec, 0, (long long)max_batch * width * g.S * sizeof(cx<float>)) != cudaSuccess) {
    cudaGetLastError();
    fno_free(f);
    delete f;
    return ACM_ERR_CUDA;
  }
  *out = f;
  return ACM_OK;
}

acm_status acm_fno_destroy(acm_fno* f) {
  if (!f) return ACM_ERR_ARG;
  if (f->st) cudaStreamSynchronize(f->st);
  else cudaDeviceSynchronize();
  fno_free(f);
  delete f;
  return ACM_OK;
}

acm_status acm_fno_num_params(acm_fno* f, long long* n) {
  if (!f || !n) return ACM_ERR_ARG;
  *n = f->np;
  return ACM_OK;
}

acm_status acm_fno_set_params(acm_fno* f, const float* theta) {
  if (!f || !theta) return ACM_ERR_ARG;
  FK(cudaMemcpyAsync(f->theta, theta, f->np * 4, cudaMemcpyDefault, f->st));
  k_f32_to_bf16<<<blocks_for(f->np), 256, 0, f->st>>>(f->theta, f->tb, f->np);
  FK(cudaGetLastError());
  FK(cudaMemsetAsync(f->m1, 0, f->np * 4, f->st));
  FK(cudaMemsetAsync(f->m2, 0, f->np * 4, f->st));
  f->step = 0;
  FK(cudaStreamSynchronize(f->st));
  return ACM_OK;
}

acm_status acm_fno_get_params(acm_fno* f, float* theta) {
  if (!f || !theta) return ACM_ERR_ARG;
  FK(cudaMemcpyAsync(theta, f->theta, f->np * 4, cudaMemcpyDefault, f->st));
  FK(cudaStreamSynchronize(f->st));
  return ACM_OK;
}

static acm_status stage_inputs(acm_fno* f, int B, const uint8_t* H, const uint8_t** Hd) {
  if (fno_on_device(H)) {
    *Hd = H;
  } else {
    FK(cudaMemcpyAsync(f->Hs, H, (size_t)B * f->d.V, cudaMemcpyHostToDevice, f->st));
    *Hd = f->Hs;
  }
  return ACM_OK;
}

acm_status acm_fno_forward(acm_fno* f, int batch, const uint8_t* H, float* out) {
  if (!f || !H || batch < 1 || batch > f->Bmax) return ACM_ERR_ARG;
  const uint8_t* Hd = nullptr;
  CKF(stage_inputs(f, batch, H, &Hd));
  float* o = out && fno_on_device(out) ? out : f->dout;
  CKF(dispatch_w(f->d.W, [&](auto w) { return fno_forward_impl<decltype(w)::value>(f, batch, Hd, nullptr, o, nullptr); }));
  if (out && o != out) FK(cudaMemcpyAsync(out, o, (size_t)batch * 6 * f->d.V * 4, cudaMemcpyDeviceToHost, f->st));
  FK(cudaStreamSynchronize(f->st));
  return ACM_OK;
}

acm_status acm_fno_warm_start(acm_fno* f, int batch, const uint8_t* H, float* init_u, float* init_lambda) {
  if (!f || !H || !init_u || !init_lambda || batch < 1 || batch > f->Bmax) return ACM_ERR_ARG;
  const Geo& g = f->g;
  if (g.n0 != g.n1 || g.n0 != g.n2) return ACM_ERR_UNSUPPORTED_SIZE;
  if (!fno_on_device(init_u) || !fno_on_device(init_lambda)) return ACM_ERR_ARG;
  const uint8_t* Hd = nullptr;
  CKF(stage_inputs(f, batch, H, &Hd));
  if (!f->Hp) FK(cudaMalloc(&f->Hp, (size_t)f->Bmax * f->d.V));
  const long long total = (long long)batch * f->d.V;
  for (int j = 0; j < 3; ++j) {
    const uint8_t* Hj = Hd;
    if (j > 0) {
      k_swap_h<<<blocks_for(total), 256, 0, f->st>>>(Hd, f->Hp, g.n0, j, f->d.V, total);
      FK(cudaGetLastError());
      Hj = f->Hp;
    }
    CKF(dispatch_w(f->d.W, [&](auto w) {
      return fno_forward_impl<decltype(w)::value>(f, batch, Hj, nullptr, f->dout, nullptr);
    }));
    k_unswap_out<<<blocks_for(total), 256, 0, f->st>>>(f->dout, init_u, init_lambda, g.n0, j, f->d.V, total);
    FK(cudaGetLastError());
  }
  FK(cudaStreamSynchronize(f->st));
  return ACM_OK;
}

acm_status acm_fno_backward(acm_fno* f, int batch, const uint8_t* H, const float* target, double* loss, float* grad) {
  if (!f || !H || !target || batch < 1 || batch > f->Bmax) return ACM_ERR_ARG;
  const uint8_t* Hd = nullptr;
  CKF(stage_inputs(f, batch, H, &Hd));
  const float* t = target;
  if (!fno_on_device(target)) {
    FK(cudaMemcpyAsync(f->tgt, target, (size_t)batch * 6 * f->d.V * 4, cudaMemcpyHostToDevice, f->st));
    t = f->tgt;
  }
  double L = 0;
  CKF(dispatch_w(f->d.W, [&](auto w) {
    acm_status s = fno_forward_impl<decltype(w)::value>(f, batch, Hd, t, nullptr, &L);
    if (s != ACM_OK) return s;
    return fno_backward_impl<decltype(w)::value>(f, batch, Hd);
  }));
  if (loss) *loss = L;
  if (grad) FK(cudaMemcpyAsync(grad, f->grad, f->np * 4, cudaMemcpyDefault, f->st));
  FK(cudaStreamSynchronize(f->st));
  return ACM_OK;
}

acm_status acm_fno_adamw(acm_fno* f, double lr, double beta1, double beta2, double eps, double weight_decay) {
  if (!f || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0) ||
      !(weight_decay >= 0))
    return ACM_ERR_ARG;
  f->step += 1;
  const float c1 = (float)(1.0 - std::pow(beta1, (double)f->step));
  const float c2 = (float)(1.0 - std::pow(beta2, (double)f->step));
  k_adamw<<<blocks_for(f->np), 256, 0, f->st>>>(f->theta, f->tb, f->grad, f->m1, f->m2, f->np, (float)lr,
                                                  (float)beta1, (float)beta2, (float)eps, (float)weight_decay, c1, c2);
  FK(cudaGetLastError());
  return ACM_OK;
}

}  // extern "C"
