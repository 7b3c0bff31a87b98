// acm_ops.h -- host-side launch wrappers of the ACM kernels (one instantiation
// per precision, compiled in separate translation units).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "acm_types.h"

namespace acm {

// P_FWD_SOL / P_INV_SOL: the y passes of the solute iteration (derivative
// terms of axis 1 folded in; see the strided kernel); P_SOLUTE: its z pass.
enum PassOp { P_FWD = 0, P_INV = 1, P_INV_SCALE = 2, P_STOKES = 3, P_SOLUTE = 4, P_DERIV = 5, P_FWD_SOL = 6,
              P_INV_SOL = 7 };

template <typename T>
struct Ops {
  // blocks per problem of the x-passes and of a z-pass (number of partial sums)
  static int x_blocks(const Geo& g);
  static int z_blocks(const Geo& g, int op);
  // tile width (columns) a strided pass launches with under g's tile choice, and
  // whether the choice `shift` (-1, 0, +1) has its own compiled variant
  static int pass_tx(const Geo& g, int axis, int op, int nc);
  static bool tx_variant(int n, int op, int nc, int shift);

  static cudaError_t x_stokes_local(const Geo& g, int nprob, const void* spec, void* u, void* lam,
                                    const uint8_t* H, const uint32_t* Hb, StokesDev* prm, double* part,
                                    const void* tw, cudaStream_t s);
  static cudaError_t x_stokes_rhs(const Geo& g, int nprob, void* spec, const void* u, const void* lam,
                                  const uint8_t* H, const uint32_t* Hb, const StokesDev* prm, const void* tw,
                                  cudaStream_t s);
  static cudaError_t x_solute(const Geo& g, int nprob, void* spec, const void* u, const uint8_t* H,
                              const uint32_t* Hb, const SoluteDev* prm, const void* tw, const Sym<T>& sym,
                              bool central, cudaStream_t s);
  // nc in {1, 3}
  static cudaError_t x_r2c(const Geo& g, int nprob, int nc, void* spec, long long specProbStride,
                           const void* in, long long inProbStride, const void* tw, cudaStream_t s);
  static cudaError_t x_c2r(const Geo& g, int nprob, int nc, const void* spec, long long specProbStride,
                           void* out, long long outProbStride, const void* tw, cudaStream_t s);
  // complex FFT pass along axis 1 (y) or 0 (z) of nc components, with operator op
  // (P_STOKES and P_SOLUTE only along z)
  static cudaError_t pass(const Geo& g, int axis, int op, int nc, int nprob, void* spec, long long probStride,
                          const Sym<T>& sym, const void* tw, void* st0, void* st1, StokesDev* sprm,
                          SoluteDev* cprm, double* part, cudaStream_t s, int dm = 0);
  // sum over pore voxels of the six products of three fields [3][V] (NRED partial records)
  static cudaError_t pore_products(const Geo& g, const void* f, const uint8_t* H, double* part, int nblk,
                                   cudaStream_t s);
  // FP64 partial sums (stride 8 doubles per block): see k_field_sums / k_diffusivity
  static cudaError_t field_sums(const Geo& g, int nprob, const void* u, const uint8_t* H, double* part, int nblk,
                                cudaStream_t s);
  static cudaError_t diffusivity(const Geo& g, int nprob, const void* chi, const void* grad, const void* u,
                                 const uint8_t* H, const SoluteDev* prm, double* part, int nblk, cudaStream_t s);
  static cudaError_t mask_solid(const Geo& g, const void* in, void* out, const uint8_t* H, cudaStream_t s);
  static cudaError_t div_spec(const Geo& g, const void* uh, void* dv, const Sym<T>& sym, cudaStream_t s);
  static cudaError_t q_from_a(const Geo& g, const void* ah, void* q, const Sym<T>& sym, cudaStream_t s);
};

// precision conversion of n elements (float <-> double)
cudaError_t convert_f2d(const float* in, double* out, long long n, cudaStream_t s);
cudaError_t convert_d2f(const double* in, float* out, long long n, cudaStream_t s);

cudaError_t stokes_finalize(int nprob, StokesDev* prm, const double* part_x, int nbx, const double* part_z,
                            int nbz, double V, double* hist, int hist_cap, cudaStream_t s);
cudaError_t solute_finalize(int nprob, SoluteDev* prm, const double* part_z, int nbz, double V, double* hist,
                            int hist_cap, cudaStream_t s);
cudaError_t count_solid(const uint8_t* H, long long V, unsigned long long* out, cudaStream_t s);
// Hb[w] = bits of H[32 w .. 32 w + 31] (n a multiple of 32)
cudaError_t pack_hbits(const uint8_t* H, uint32_t* Hb, long long n, cudaStream_t s);
cudaError_t count_solid_add(const uint8_t* H, long long V, unsigned long long* out, cudaStream_t s);
// adds the number of solid-pore faces of H (periodic) to *out
cudaError_t count_faces_add(const uint8_t* H, int n0, int n1, int n2, unsigned long long* out, cudaStream_t s);

// Condition of the device-resident loop (a CUDA graph while node): continue
// while any problem of any group has not set its stop flag, and at most `cap`
// iterations. Group g has n[g] control blocks of `stride` bytes starting at
// base[g]; the stop flag is the int at byte offset `done_off` of each block.
struct LoopCtl {
  const char* base[4];
  int n[4];
  int stride[4];
  int ngroups;
  int done_off;
  unsigned int* counter;  // iterations run so far (device)
  unsigned int cap;
  cudaGraphConditionalHandle handle;
};
cudaError_t loop_control(const LoopCtl& c, cudaStream_t s);

}  // namespace acm
