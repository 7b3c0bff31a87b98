// acm_misc.cu -- precision-independent kernels: FP64 finalize steps of both
// iterations, precision conversion and the solid-voxel count.
#include "acm_fft.cuh"
#include "acm_kernels.cuh"
#include "acm_ops.h"

namespace acm {
// ---------------------------------------------------------------------------
// finalize kernels: deterministic FP64 sums of the partials, Eq. 10-12, Eq. 22
// ---------------------------------------------------------------------------
__device__ __forceinline__ void sum_partials(const double* __restrict__ part, int nblk, int stride, int nval,
                                             double* out, double* red) {
  double acc[5] = {0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < nblk; i += blockDim.x)
    for (int k = 0; k < nval; ++k) acc[k] += part[(long long)i * stride + k];
  block_sum_store<5>(acc, red, out);
  __syncthreads();
}

// Stagnation test of an FP32 phase (off when win = 0): the distance to the
// tolerance m = max_k r[k] / t[k] must fall below STALL_DROP times its best
// value within `win` iterations, else the phase has reached its rounding floor.
__device__ __forceinline__ bool stalled(int win, int& n, double& best, const double* r, const double* t, int k) {
  if (win <= 0) return false;
  double m = 0.0;
  for (int i = 0; i < k; ++i) m = fmax(m, t[i] > 0.0 ? r[i] / t[i] : r[i]);
  if (m < STALL_DROP * best) {
    best = m;
    n = 0;
    return false;
  }
  return ++n >= win;
}

__global__ void __launch_bounds__(256) k_stokes_finalize(StokesDev* __restrict__ prm, const double* __restrict__ part_x,
                                                        int nbx, const double* __restrict__ part_z, int nbz,
                                                        double V, double* __restrict__ hist, int hist_cap) {
  __shared__ double red[5 * 32];
  __shared__ double sx[5], sz[5];
  const int p = blockIdx.x;
  StokesDev* P = prm + p;
  if (P->done) return;
  sum_partials(part_x + (long long)p * nbx * 8, nbx, 8, 5, sx, red);
  sum_partials(part_z + (long long)p * nbz * 4, nbz, 4, 3, sz, red);
  if (threadIdx.x != 0) return;
  const double alpha = P->psi[0], beta = P->psi[1], b = P->psi[2];
  double r[6];
  r[0] = sqrt(sx[0]);
  r[1] = alpha * sqrt(sx[1]);
  r[2] = sqrt(sz[0] / V);
  r[3] = beta * sqrt(sz[1] / V);
  r[4] = sqrt(sx[2]);
  r[5] = b * sqrt(sx[3]);
  const double nl = sqrt(sx[4]), nq = sqrt(sz[2] / V), na = nl;  // a = H lambda
  const double e = P->eps, s13 = sqrt(3.0 * V) * e, s2 = sqrt(V) * e;
  double t[6];
  t[0] = s13 + e * fmax(r[0], nl);
  t[1] = s13 + e * nl;
  t[2] = s2 + e * fmax(r[2], nq);
  t[3] = s2 + e * nq;
  t[4] = s13 + e * fmax(r[4], na);
  t[5] = s13 + e * na;
  bool conv = true, finite = true;
  for (int k = 0; k < 6; ++k) {
    P->res[k] = r[k];
    P->tol[k] = t[k];
    conv = conv && (r[k] <= t[k]);
    finite = finite && isfinite(r[k]);
  }
  P->iter += 1;
  const int it = P->iter;
  if (hist && it + P->iter_base <= hist_cap) {
    double* h = hist + ((long long)p * hist_cap + (it + P->iter_base - 1)) * STOKES_HIST;
    for (int k = 0; k < 6; ++k) h[k] = r[k];
    for (int k = 0; k < 6; ++k) h[6 + k] = t[k];
    h[12] = alpha;
    h[13] = beta;
    h[14] = b;
    for (int k = 0; k < 3; ++k) h[15 + k] = P->mean_u[k];
    h[18] = 0.0;
    h[19] = 0.0;
  }
  for (int k = 0; k < 3; ++k) {
    P->psi_last[k] = P->psi[k];
    P->psi_prev[k] = P->psi[k];
  }
  if (P->adaptive) {
    for (int k = 0; k < 3; ++k) {  // Eq. 22: pair k drives (alpha, beta, b)[k]
      const double rp = r[2 * k], rd = r[2 * k + 1];
      if (rp > P->tau[k] * rd) P->psi[k] = P->phi[k] * P->psi[k];
      else if (rd > P->tau[k] * rp) P->psi[k] = fmax(P->psi[k] / P->phi[k], P->psi_min[k]);
    }
  }
  if (!finite) {
    P->done = 1;
    P->status = ST_NONFINITE;
  } else if (conv) {
    P->done = 1;
    P->converged = 1;
    P->status = ST_OK;
  } else if (stalled(P->stall_win, P->stall_n, P->stall_best, r, t, 6)) {
    P->done = 1;
    P->status = ST_STALLED;
  } else if (it >= P->max_iter) {
    P->done = 1;
    P->status = ST_MAXITER;
  }
}

__global__ void __launch_bounds__(256) k_solute_finalize(SoluteDev* __restrict__ prm, const double* __restrict__ part_z,
                                                        int nbz, double V, double* __restrict__ hist, int hist_cap) {
  __shared__ double red[5 * 32];
  __shared__ double sz[5];
  const int p = blockIdx.x;
  SoluteDev* P = prm + p;
  if (P->done) return;
  sum_partials(part_z + (long long)p * nbz * 4, nbz, 4, 2, sz, red);
  if (threadIdx.x != 0) return;
  const double r1 = sqrt(sz[0] / V), r2 = sqrt(sz[1] / V);
  const double t1 = sqrt(V) * P->eps, t2 = sqrt(3.0 * V) * P->eps;
  P->res[0] = r1;
  P->res[1] = r2;
  P->tol[0] = t1;
  P->tol[1] = t2;
  P->iter += 1;
  const int it = P->iter;
  if (hist && it + P->iter_base <= hist_cap) {
    double* h = hist + ((long long)p * hist_cap + (it + P->iter_base - 1)) * SOLUTE_HIST;
    h[0] = r1;
    h[1] = r2;
    h[2] = t1;
    h[3] = t2;
  }
  const double rn = r1 / (1.0 + t1);
  if (!(isfinite(r1) && isfinite(r2))) {
    P->done = 1;
    P->status = ST_NONFINITE;
    return;
  }
  if (r1 <= t1 && r2 <= t2) {
    P->done = 1;
    P->converged = 1;
    P->status = ST_OK;
    return;
  }
  if (it > 20 && rn > 1e3 * P->rmin) {
    P->done = 1;
    P->status = ST_DIVERGED;
    return;
  }
  if (rn < P->rmin) P->rmin = rn;
  const double rr[2] = {r1, r2}, tt[2] = {t1, t2};
  if (stalled(P->stall_win, P->stall_n, P->stall_best, rr, tt, 2)) {
    P->done = 1;
    P->status = ST_STALLED;
    return;
  }
  if (it >= P->max_iter) {
    P->done = 1;
    P->status = ST_MAXITER;
  }
}

// solid-pore faces of the periodic voxel grid: each voxel counts the faces it
// shares with its +1 neighbours along the three axes where H changes (a grid of
// one plane has no face along axis 0)
__global__ void k_count_faces(const uint8_t* __restrict__ H, int n0, int n1, int n2, unsigned long long* out) {
  const long long V = (long long)n0 * n1 * n2;
  unsigned long long c = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
    const int i2 = (int)(i % n2);
    const long long r = i / n2;
    const int i1 = (int)(r % n1), i0 = (int)(r / n1);
    const uint8_t h = H[i] != 0;
    const long long a0 = ((long long)((i0 + 1) % n0) * n1 + i1) * n2 + i2;
    const long long a1 = ((long long)i0 * n1 + (i1 + 1) % n1) * n2 + i2;
    const long long a2 = ((long long)i0 * n1 + i1) * n2 + (i2 + 1) % n2;
    c += (unsigned long long)(h != (H[a0] != 0)) + (h != (H[a1] != 0)) + (h != (H[a2] != 0));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

__global__ void k_count_solid(const uint8_t* __restrict__ H, long long V, unsigned long long* out) {
  unsigned long long c = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x)
    c += H[i] ? 1ull : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

__global__ void __launch_bounds__(256) k_loop_control(LoopCtl c) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  int mine = 0;
  for (int gi = 0; gi < c.ngroups; ++gi)
    for (int i = threadIdx.x; i < c.n[gi]; i += blockDim.x)
      mine |= (*reinterpret_cast<const int*>(c.base[gi] + (size_t)i * c.stride[gi] + c.done_off) == 0);
  if (mine) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int it = *c.counter + 1;
    *c.counter = it;
    cudaGraphSetConditional(c.handle, (any && it < c.cap) ? 1u : 0u);
  }
}

cudaError_t loop_control(const LoopCtl& c, cudaStream_t s) {
  k_loop_control<<<1, 256, 0, s>>>(c);
  return cudaGetLastError();
}

cudaError_t stokes_finalize(int nprob, StokesDev* prm, const double* part_x, int nbx, const double* part_z,
                            int nbz, double V, double* hist, int hist_cap, cudaStream_t s) {
  k_stokes_finalize<<<nprob, 256, 0, s>>>(prm, part_x, nbx, part_z, nbz, V, hist, hist_cap);
  return cudaGetLastError();
}

cudaError_t solute_finalize(int nprob, SoluteDev* prm, const double* part_z, int nbz, double V, double* hist,
                            int hist_cap, cudaStream_t s) {
  k_solute_finalize<<<nprob, 256, 0, s>>>(prm, part_z, nbz, V, hist, hist_cap);
  return cudaGetLastError();
}

// one bit per voxel of H: word w holds voxels 32 w .. 32 w + 31 (n a multiple of
// 32, so every warp of the grid-stride loop sees 32 valid voxels)
__global__ void k_hbits(const uint8_t* __restrict__ H, uint32_t* __restrict__ Hb, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned b = __ballot_sync(0xffffffffu, H[i] != 0);
    if ((threadIdx.x & 31) == 0) Hb[i >> 5] = b;
  }
}

cudaError_t pack_hbits(const uint8_t* H, uint32_t* Hb, long long n, cudaStream_t s) {
  if (n % 32 != 0) return cudaErrorInvalidValue;
  k_hbits<<<608, 256, 0, s>>>(H, Hb, n);
  return cudaGetLastError();
}

cudaError_t count_solid(const uint8_t* H, long long V, unsigned long long* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_count_solid<<<304, 256, 0, s>>>(H, V, out);
  return cudaGetLastError();
}

cudaError_t count_faces_add(const uint8_t* H, int n0, int n1, int n2, unsigned long long* out, cudaStream_t s) {
  k_count_faces<<<304, 256, 0, s>>>(H, n0, n1, n2, out);
  return cudaGetLastError();
}

cudaError_t count_solid_add(const uint8_t* H, long long V, unsigned long long* out, cudaStream_t s) {
  k_count_solid<<<304, 256, 0, s>>>(H, V, out);
  return cudaGetLastError();
}

cudaError_t convert_f2d(const float* in, double* out, long long n, cudaStream_t s) {
  k_convert<float, double><<<608, 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t convert_d2f(const double* in, float* out, long long n, cudaStream_t s) {
  k_convert<double, float><<<608, 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

}  // namespace acm
