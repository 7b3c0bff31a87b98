// acm_types.h -- plain data shared by the host driver and the device kernels.
#pragma once

namespace acm {

constexpr int STOKES_HIST = 20;  // doubles per Stokes history record
constexpr int SOLUTE_HIST = 4;   // doubles per solute history record

constexpr int TW_MAX = 1024;  // master twiddle table length (>= 2 * the largest axis)

// ---------------------------------------------------------------------------
// device-side per-problem state of a solve
// ---------------------------------------------------------------------------
struct StokesDev {
  // set by the host before the solve
  double nu, eps, g[3];
  double phi[3], tau[3], psi_min[3];
  int adaptive, max_iter;
  // evolving
  double psi[3];       // alpha, beta, b used by the coming iteration
  double psi_prev[3];  // penalties of the iteration that produced the stored u
  double psi_last[3];  // penalties of the last finalised iteration
  double res[6], tol[6];
  double mean_u[3];    // k = 0 tap of the last Green step (volume average of u)
  int iter, done, status, converged;
  int iter_base;       // iterations of earlier phases (history indexing)
  // stagnation of an FP32 phase (stall_win > 0): the solve stops with
  // ST_STALLED when max_k res[k] / tol[k] has not fallen below STALL_DROP times
  // its best value for stall_win iterations (its FP32 rounding floor)
  int stall_win, stall_n;
  double stall_best;
};

struct SoluteDev {
  double eps, A0, eta, Pe;
  double B0[3], g[3], ubar[3];
  double Fc;           // Pe * ubar . g
  int max_iter;
  double res[2], tol[2];
  double rmin;
  int iter, done, status, converged;
  int iter_base;
  int stall_win, stall_n;  // as in StokesDev
  double stall_best;
};

// improvement factor that resets the stagnation count of an FP32 phase
constexpr double STALL_DROP = 0.98;

// status codes mirrored from acm.h
enum { ST_OK = 0, ST_MAXITER = -4, ST_DIVERGED = -5, ST_NONFINITE = -6 };
// internal: an FP32 phase stopped at its rounding floor (the driver continues
// that problem in FP64; never returned to the caller)
enum { ST_STALLED = -100 };

// Geometry of one grid and its half spectrum.
struct Geo {
  int n0, n1, n2;
  int P;        // row pitch of the half spectrum (complex elements), >= n2/2 + 1
  int Pu;       // used columns n2/2 + 1
  long long V;  // voxels
  long long S;  // complex elements of one spectral component: n0 * n1 * P
  long long hs; // stride of H between problems of a batch (0: one shared H)
  long long us; // stride of the advecting velocity between problems (0: shared)
  int lph;      // problems per indicator: problem p uses H + (p / lph) * hs
  // tile-width choice of the strided passes per [precision (FP64 = 1)][axis][pass op]:
  // -1 half, 0 default, +1 double, +2 four times the default width (set by the autotuner)
  signed char txs[2][2][8] = {};
};

// Symbols of one precision: d and L per axis (axis 2 only up to n2/2).
template <typename T>
struct Sym {
  const T* d0;
  const T* l0;
  const T* d1;
  const T* l1;
  const T* d2;
  const T* l2;
};

}  // namespace acm
