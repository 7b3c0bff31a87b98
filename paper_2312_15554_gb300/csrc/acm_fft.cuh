// acm_fft.cuh -- shared-memory Stockham FFT building blocks for sm_103a.
//
// Every 1D transform of length N runs on one "line" held in shared memory.
// A line is processed by T = N / E threads of one warp (E = elements per
// thread, at most 16), so the stages synchronise with __syncwarp only.
// Each stage reads E values into registers, applies the twiddles and an
// in-register DFT of radix R (R divides E), and writes the results back in
// Stockham (self-sorting) order, so the output is in natural order.
//
// Shared-memory lines are padded with one slot per 16 elements (pad()) so that
// the stride-R writes of the first stage and the transposed tile loads of the
// strided passes spread over all banks.
//
// The forward transform uses exp(-2 pi i k n / N) and is unnormalised; the
// inverse uses exp(+2 pi i k n / N) and is unnormalised too.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace acm {

template <typename T>
struct __align__(2 * sizeof(T)) cx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cx<T> mk(T a, T b) {
  cx<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ cx<T> cconj(cx<T> a) { return mk<T>(a.x, -a.y); }
template <typename T>
__device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// i * a
template <typename T>
__device__ __forceinline__ cx<T> mul_i(cx<T> a) { return mk<T>(-a.y, a.x); }
template <typename T>
__device__ __forceinline__ T cabs2(cx<T> a) { return a.x * a.x + a.y * a.y; }

// padded shared-memory index: one spare slot after every 16 elements
__host__ __device__ constexpr int pad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int ept(int n) { return n < 16 ? n : 16; }  // elements per thread

// Stride (complex elements) between padded lines of length L in shared memory.
// One shared-memory wavefront serves W = 128 bytes / element size threads (16
// for FP32 complex, 8 for FP64 complex), each touching one slot. When a line's
// transform uses TL < W threads, a wavefront spans W/TL lines and each line
// covers TL consecutive slots, so the lines must start TL slots apart modulo W:
// stride = TL * odd (mod W). When lines are loaded as the TX columns of a tile
// (TX threads per row, W/TX rows per wavefront) the columns must start W/TX
// slots apart. The first stride at or above the padded length that meets the
// active constraint is used; with TL < W the transform's constraint wins (it
// is accessed more often).
__host__ __device__ constexpr int line_stride(int L, int TL, int TX, int W) {
  int ls = (L - 1) + ((L - 1) >> 4) + 1;
  const int q = TL < W ? TL : (TX >= 1 && TX < W ? W / TX : 1);
  while (((ls / q) % 2) == 0 || (ls % q) != 0) ++ls;
  return ls;
}

template <typename T>
__host__ __device__ constexpr int wave_slots() { return 128 / (2 * (int)sizeof(T)); }

// multiply by exp(SIGN * i * pi / 2): SIGN = -1 -> -i, SIGN = +1 -> +i
template <int SIGN, typename T>
__device__ __forceinline__ cx<T> rot4(cx<T> a) {
  return SIGN < 0 ? mk<T>(a.y, -a.x) : mk<T>(-a.y, a.x);
}

// multiply by W16^m = exp(SIGN * 2 pi i m / 16) for compile-time m
template <int SIGN, int M, typename T>
__device__ __forceinline__ cx<T> tw16(cx<T> a) {
  constexpr int m = M & 15;
  if constexpr (m == 0) {
    return a;
  } else if constexpr (m == 4) {
    return rot4<SIGN>(a);
  } else if constexpr (m == 8) {
    return mk<T>(-a.x, -a.y);
  } else if constexpr (m == 12) {
    return rot4<-SIGN>(a);
  } else {
    // cos and sin of m * pi / 8 for m in {1, 2, 3, 5, 6, 7, 9, ...}
    constexpr double C1 = 0.92387953251128675613, S1 = 0.38268343236508977173;
    constexpr double C2 = 0.70710678118654752440;
    constexpr double cs[16] = {1.0, C1, C2, S1, 0.0, -S1, -C2, -C1, -1.0, -C1, -C2, -S1, 0.0, S1, C2, C1};
    constexpr double sn[16] = {0.0, S1, C2, C1, 1.0, C1, C2, S1, 0.0, -S1, -C2, -C1, -1.0, -C1, -C2, -S1};
    const T c = (T)cs[m];
    const T s = (T)(SIGN * sn[m]);
    return mk<T>(a.x * c - a.y * s, a.x * s + a.y * c);
  }
}

// multiply by W32^m = exp(SIGN * 2 pi i m / 32) for compile-time m
template <int SIGN, int M, typename T>
__device__ __forceinline__ cx<T> tw32(cx<T> a) {
  constexpr int m = M & 31;
  if constexpr (m % 2 == 0) {
    return tw16<SIGN, m / 2>(a);
  } else {
    // cos and sin of m * pi / 16 for odd m < 16; m + 16 is the negation
    constexpr double C1 = 0.98078528040323044913, S1 = 0.19509032201612826785;
    constexpr double C3 = 0.83146961230254523708, S3 = 0.55557023301960222474;
    constexpr double cs[8] = {C1, C3, S3, S1, -S1, -S3, -C3, -C1};
    constexpr double sn[8] = {S1, S3, C3, C1, C1, C3, S3, S1};
    constexpr double neg = m > 16 ? -1.0 : 1.0;
    const T c = (T)(neg * cs[(m & 15) / 2]);
    const T s = (T)(SIGN * neg * sn[(m & 15) / 2]);
    return mk<T>(a.x * c - a.y * s, a.x * s + a.y * c);
  }
}

// multiply by exp(SIGN * 2 pi i m / R) for compile-time m and R in {1, 2, 4, 8, 16, 32}
template <int SIGN, int M, int R, typename T>
__device__ __forceinline__ cx<T> root_mul(cx<T> a) {
  static_assert(R >= 1 && R <= 32 && (R & (R - 1)) == 0, "R must be a power of two up to 32");
  return tw32<SIGN, M * (32 / R)>(a);
}

// f(ic<i>{}) for i = 0..N-1: inside f, decltype(arg)::value is the constant expression i
template <int I>
struct ic {
  static constexpr int value = I;
};
template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(ic<I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// ---------------------------------------------------------------------------
// in-register DFTs of radix 2, 4, 8, 16 (natural-order in and out)
// ---------------------------------------------------------------------------
template <int SIGN, typename T>
__device__ __forceinline__ void dft2(cx<T>* v) {
  cx<T> a = v[0];
  v[0] = a + v[1];
  v[1] = a - v[1];
}

template <int SIGN, typename T>
__device__ __forceinline__ void dft4(cx<T>& v0, cx<T>& v1, cx<T>& v2, cx<T>& v3) {
  cx<T> t0 = v0 + v2, t1 = v0 - v2, t2 = v1 + v3, t3 = rot4<SIGN>(v1 - v3);
  v0 = t0 + t2;
  v2 = t0 - t2;
  v1 = t1 + t3;
  v3 = t1 - t3;
}

template <int SIGN, typename T>
__device__ __forceinline__ void dft4(cx<T>* v) { dft4<SIGN>(v[0], v[1], v[2], v[3]); }

template <int SIGN, typename T>
__device__ __forceinline__ void dft8(cx<T>* v) {
  cx<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  cx<T> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<SIGN>(e0, e1, e2, e3);
  dft4<SIGN>(o0, o1, o2, o3);
  o1 = tw16<SIGN, 2>(o1);
  o2 = tw16<SIGN, 4>(o2);
  o3 = tw16<SIGN, 6>(o3);
  v[0] = e0 + o0;
  v[4] = e0 - o0;
  v[1] = e1 + o1;
  v[5] = e1 - o1;
  v[2] = e2 + o2;
  v[6] = e2 - o2;
  v[3] = e3 + o3;
  v[7] = e3 - o3;
}

template <int SIGN, typename T>
__device__ __forceinline__ void dft16(cx<T>* v) {
  // n = 4 n1 + n2, k = k1 + 4 k2
  cx<T> y[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    y[n2][0] = v[n2];
    y[n2][1] = v[4 + n2];
    y[n2][2] = v[8 + n2];
    y[n2][3] = v[12 + n2];
    dft4<SIGN>(y[n2][0], y[n2][1], y[n2][2], y[n2][3]);
  }
  y[1][1] = tw16<SIGN, 1>(y[1][1]);
  y[1][2] = tw16<SIGN, 2>(y[1][2]);
  y[1][3] = tw16<SIGN, 3>(y[1][3]);
  y[2][1] = tw16<SIGN, 2>(y[2][1]);
  y[2][2] = tw16<SIGN, 4>(y[2][2]);
  y[2][3] = tw16<SIGN, 6>(y[2][3]);
  y[3][1] = tw16<SIGN, 3>(y[3][1]);
  y[3][2] = tw16<SIGN, 6>(y[3][2]);
  y[3][3] = tw16<SIGN, 9>(y[3][3]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    cx<T> a = y[0][k1], b = y[1][k1], c = y[2][k1], d = y[3][k1];
    dft4<SIGN>(a, b, c, d);
    v[k1] = a;
    v[k1 + 4] = b;
    v[k1 + 8] = c;
    v[k1 + 12] = d;
  }
}

template <int R, int SIGN, typename T>
__device__ __forceinline__ void dft(cx<T>* v) {
  if constexpr (R == 2) dft2<SIGN>(v);
  else if constexpr (R == 4) dft4<SIGN>(v);
  else if constexpr (R == 8) dft8<SIGN>(v);
  else if constexpr (R == 16) dft16<SIGN>(v);
}

// ---------------------------------------------------------------------------
// Stage twiddles. The stage that starts at span Ns (> 1) with radix R needs
// W_N^{jm r N / (Ns R)} for r in [1, R) and jm in [0, Ns); they are stored as
// [r - 1][jm] so that the threads of a line read consecutive entries.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int stage_radix(int N, int Ns) { return (N / Ns >= ept(N)) ? ept(N) : N / Ns; }

__host__ __device__ constexpr int tw_offset(int N, int Ns) {
  int off = 0;
  for (int s = 1; s < Ns; s *= stage_radix(N, s))
    if (s > 1) off += (stage_radix(N, s) - 1) * s;
  return off;
}

__host__ __device__ constexpr int tw_total(int N) { return tw_offset(N, N) > 0 ? tw_offset(N, N) : 1; }

// fill the stage tables of a length-N transform from W_TWM^k, k < TWM (TWM a multiple of N)
template <typename T, int N, int Ns, int TWM>
struct FillTw {
  static __device__ __forceinline__ void run(cx<T>* tw, const cx<T>* __restrict__ master) {
    if constexpr (Ns < N) {
      constexpr int R = stage_radix(N, Ns);
      if constexpr (Ns > 1) {
        constexpr int off = tw_offset(N, Ns);
        for (int e = threadIdx.x; e < (R - 1) * Ns; e += blockDim.x) {
          const int r = e / Ns + 1, jm = e - (r - 1) * Ns;
          tw[off + e] = master[(jm * r * (N / (Ns * R))) * (TWM / N)];
        }
      }
      FillTw<T, N, Ns * R, TWM>::run(tw, master);
    }
  }
};

// ---------------------------------------------------------------------------
// Stockham stage: radix R, Ns = product of the previous radices
// tw: the per-stage twiddle tables of this transform length (see FillTw)
// ---------------------------------------------------------------------------
template <typename T, int N, int R, int Ns, int SIGN>
__device__ __forceinline__ void stockham_stage(cx<T>* s, int t, const cx<T>* __restrict__ tw, unsigned mask) {
  constexpr int E = ept(N);
  constexpr int TT = N / E;
  constexpr int NB = E / R;
  cx<T> v[NB][R];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int j = t + i * TT;
#pragma unroll
    for (int r = 0; r < R; ++r) v[i][r] = s[pad(j + r * (N / R))];
  }
  if constexpr (TT > 1) __syncwarp(mask);
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int j = t + i * TT;
    const int jm = j & (Ns - 1);
    if constexpr (Ns > 1) {
      const cx<T>* tws = tw + tw_offset(N, Ns) + jm;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cx<T> w = tws[(r - 1) * Ns];
        if constexpr (SIGN > 0) w.y = -w.y;
        v[i][r] = cmul(v[i][r], w);
      }
    }
    dft<R, SIGN>(v[i]);
    const int base = (j - jm) * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) s[pad(base + r * Ns)] = v[i][r];
  }
  if constexpr (TT > 1) __syncwarp(mask);
}

template <typename T, int N, int Ns, int SIGN>
struct Stockham {
  static __device__ __forceinline__ void run(cx<T>* s, int t, const cx<T>* tw, unsigned mask) {
    if constexpr (Ns < N) {
      constexpr int R = stage_radix(N, Ns);
      stockham_stage<T, N, R, Ns, SIGN>(s, t, tw, mask);
      Stockham<T, N, Ns * R, SIGN>::run(s, t, tw, mask);
    }
  }
};

// Transform one padded shared-memory line of length N with thread t of N/E.
// mask: the lanes of the calling warp that are transforming lines (each line's
// N/E threads are consecutive lanes of one warp).
template <typename T, int N, int SIGN>
__device__ __forceinline__ void fft_line(cx<T>* s, int t, const cx<T>* tw, unsigned mask) {
  Stockham<T, N, 1, SIGN>::run(s, t, tw, mask);
}

// ---------------------------------------------------------------------------
// asynchronous global -> shared copies (cp.async): the loads of a tile are all
// in flight at once and do not pass through registers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async size");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_u32(smem)), "l"(gmem), "n"(BYTES));
}

// copy BYTES when pred, else write zeros to shared memory (no global access)
template <int BYTES>
__device__ __forceinline__ void cp_async_pred(void* smem, const void* gmem, bool pred) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_u32(smem)), "l"(gmem), "n"(BYTES),
               "r"(pred ? BYTES : 0));
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }

// Bulk prefetch of bytes (a multiple of 16, 16-byte aligned, in bounds) into L2.
__device__ __forceinline__ void prefetch_l2(const void* gmem, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(gmem), "r"(bytes) : "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of NS values per thread, written by thread 0 to out[0..NS) as
// doubles. The warp and block stages run in T: FP32 kernels sum their block's
// few hundred partials in FP32 (FP64 arithmetic is scarce on this GPU) and
// hand FP64 on to the grid stage. scratch: NS * 32 values of T in shared
// memory. Deterministic for a fixed block size.
template <int NS, typename T>
__device__ __forceinline__ void block_sum_store(T (&v)[NS], T* scratch, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NS; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NS; ++k) scratch[k * 32 + warp] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      T a = lane < nw ? scratch[k * 32 + lane] : (T)0;
      a = warp_sum(a);
      if (lane == 0) out[k] = (double)a;
    }
  }
}

}  // namespace acm
