/*
 * oracle_fft.c -- the oracle's own discrete Fourier transform (test
 * infrastructure only; nothing in the product library links or calls it).
 *
 * The method of the paper moves every field between real and Fourier space
 * (Algorithm 1; Eq. 13 and Eq. 20 are solved per wavevector). The oracle does
 * the same with this plain transform:
 *
 *   forward  X[m] = sum_{j=0}^{n-1} x[j] exp(-2 pi i j m / n)      (sign = -1)
 *   inverse  x[j] = sum_{m=0}^{n-1} X[m] exp(+2 pi i j m / n)      (sign = +1,
 *            unnormalised; the caller divides by n)
 *
 * computed, when n is a power of two, with the iterative radix-2 Cooley-Tukey
 * algorithm: the input is put in bit-reversed order, then log2(n) stages of
 * butterflies combine transforms of length 2s from pairs of length s. Every
 * twiddle exp(sign 2 pi i k / 2s) is evaluated directly with cos and sin (no
 * recurrence), so the rounding error stays at a few ulps times log2(n). Other
 * lengths (small test grids only) take the O(n^2) sum above, with the phase
 * j m reduced modulo n in integer arithmetic.
 *
 * oracle_fft_axis transforms every line of one axis of a C-contiguous array of
 * complex doubles (interleaved re, im) viewed as [outer][n][inner]: line (o, i)
 * holds the elements o*n*inner + j*inner + i, j = 0..n-1. Lines are gathered
 * in blocks of up to 16 consecutive inner indices (so each read touches whole
 * cache lines), transformed one by one and scattered back. OpenMP spreads the
 * blocks over the host cores when the library is built with -fopenmp.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define BLK 16

static const double TWO_PI = 6.283185307179586476925286766559;

/* in-place radix-2 transform of one contiguous line of n = 2^p complex values */
static void fft_line(double* x, int n, int sign) {
  /* bit-reversal permutation */
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j |= bit;
    if (i < j) {
      double tr = x[2 * i], ti = x[2 * i + 1];
      x[2 * i] = x[2 * j];
      x[2 * i + 1] = x[2 * j + 1];
      x[2 * j] = tr;
      x[2 * j + 1] = ti;
    }
  }
  /* butterflies: transforms of length 2s from pairs of length s */
  for (int s = 1; s < n; s <<= 1) {
    for (int k = 0; k < s; ++k) {
      const double ang = sign * TWO_PI * (double)k / (double)(2 * s);
      const double wr = cos(ang), wi = sin(ang);
      for (int b = 0; b < n; b += 2 * s) {
        double* e = x + 2 * (b + k);
        double* o = x + 2 * (b + k + s);
        const double tr = wr * o[0] - wi * o[1];
        const double ti = wr * o[1] + wi * o[0];
        o[0] = e[0] - tr;
        o[1] = e[1] - ti;
        e[0] += tr;
        e[1] += ti;
      }
    }
  }
}

/* the sum of the definition for one line of any length n (scratch: 2n doubles) */
static void dft_line(double* x, int n, int sign, double* scratch) {
  for (int m = 0; m < n; ++m) {
    double re = 0.0, im = 0.0;
    for (int j = 0; j < n; ++j) {
      const long long ph = ((long long)j * m) % n;
      const double ang = sign * TWO_PI * (double)ph / (double)n;
      const double c = cos(ang), s = sin(ang);
      re += x[2 * j] * c - x[2 * j + 1] * s;
      im += x[2 * j] * s + x[2 * j + 1] * c;
    }
    scratch[2 * m] = re;
    scratch[2 * m + 1] = im;
  }
  memcpy(x, scratch, sizeof(double) * 2 * (size_t)n);
}

/* Returns 0 on success, -1 when n < 1 or an allocation fails. */
int oracle_fft_axis(double* data, long long outer, int n, long long inner, int sign) {
  if (n < 1) return -1;
  if (n == 1) return 0;
  const int pow2 = (n & (n - 1)) == 0;
  const long long nblk_inner = (inner + BLK - 1) / BLK;
  const long long nblk = outer * nblk_inner;
  int fail = 0;
#pragma omp parallel
  {
    /* every thread reaches the worksharing loop, with or without a buffer */
    double* buf = (double*)malloc(sizeof(double) * 2 * (size_t)n * (BLK + 1));
    if (!buf) {
#pragma omp atomic write
      fail = 1;
    }
#pragma omp for schedule(static)
    for (long long b = 0; b < nblk; ++b) {
      if (!buf) continue;
      const long long o = b / nblk_inner;
      const long long i0 = (b % nblk_inner) * BLK;
      const int w = (int)((inner - i0) < BLK ? (inner - i0) : BLK);
      double* base = data + 2 * (o * (long long)n * inner + i0);
      /* gather w lines, each contiguous in buf */
      for (int j = 0; j < n; ++j) {
        const double* src = base + 2 * (long long)j * inner;
        for (int c = 0; c < w; ++c) {
          buf[2 * ((long long)c * n + j)] = src[2 * c];
          buf[2 * ((long long)c * n + j) + 1] = src[2 * c + 1];
        }
      }
      for (int c = 0; c < w; ++c) {
        if (pow2)
          fft_line(buf + 2 * (long long)c * n, n, sign);
        else
          dft_line(buf + 2 * (long long)c * n, n, sign, buf + 2 * (long long)BLK * n);
      }
      for (int j = 0; j < n; ++j) {
        double* dst = base + 2 * (long long)j * inner;
        for (int c = 0; c < w; ++c) {
          dst[2 * c] = buf[2 * ((long long)c * n + j)];
          dst[2 * c + 1] = buf[2 * ((long long)c * n + j) + 1];
        }
      }
    }
    free(buf);
  }
  return fail ? -1 : 0;
}

/* threads the transforms use (1 without OpenMP) */
int oracle_fft_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
