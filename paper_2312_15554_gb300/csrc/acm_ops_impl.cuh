// acm_ops_impl.cuh -- definitions of the launch wrappers; included once per
// precision (acm_f32.cu, acm_f64.cu) followed by an explicit instantiation.
#pragma once
#include <cstdlib>

#include "acm_kernels.cuh"
#include "acm_ops.h"

namespace acm {

// Tile width (kx columns) of a strided pass: about 256 threads per block (many
// resident blocks hide the memory latency better than wide tiles), at least 2
// columns, and at most 64 KB of shared memory.
constexpr int pick_tx(int csize, int N, int NC) {
  int tl = N / ept(N);
  int tx = 16;
  while (tx > 2 && (NC * tx * tl > 256 || NC * tx * line_stride(N, tl, tx, 128 / csize) * csize > 64 * 1024)) tx /= 2;
  return tx;
}

template <typename K>
static cudaError_t set_smem(K* k, int bytes) {
  return bytes > 48 * 1024 ? cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
                           : cudaSuccess;
}

// the strided passes also take lines of one point (axis 0 of a single plane):
// the transform is the identity and the pass applies its operator
#define ACM_DISPATCH_NS(n, FN, ...)             \
  switch (n) {                                  \
    case 1: return FN<T, 1>(__VA_ARGS__);       \
    case 8: return FN<T, 8>(__VA_ARGS__);       \
    case 16: return FN<T, 16>(__VA_ARGS__);     \
    case 32: return FN<T, 32>(__VA_ARGS__);     \
    case 64: return FN<T, 64>(__VA_ARGS__);     \
    case 128: return FN<T, 128>(__VA_ARGS__);   \
    case 256: return FN<T, 256>(__VA_ARGS__);   \
    case 512: return FN<T, 512>(__VA_ARGS__);   \
    default: return cudaErrorInvalidValue;      \
  }

#define ACM_DISPATCH_N(n, FN, ...)     \
  switch (n) {                         \
    case 8: return FN<T, 8>(__VA_ARGS__);     \
    case 16: return FN<T, 16>(__VA_ARGS__);   \
    case 32: return FN<T, 32>(__VA_ARGS__);   \
    case 64: return FN<T, 64>(__VA_ARGS__);   \
    case 128: return FN<T, 128>(__VA_ARGS__); \
    case 256: return FN<T, 256>(__VA_ARGS__); \
    case 512: return FN<T, 512>(__VA_ARGS__); \
    default: return cudaErrorInvalidValue;    \
  }

template <typename T, int N2>
static cudaError_t l_x_local(const Geo& g, int nprob, const void* spec, void* u, void* lam, const uint8_t* H,
                             const uint32_t* Hb, StokesDev* prm, double* part, const void* tw, cudaStream_t s) {
  constexpr int smem = xs_smem_bytes<T, N2, 2, 0>();
  static const cudaError_t attr = set_smem(k_x_stokes_local<T, N2>, smem);
  if (attr != cudaSuccess) return attr;
  dim3 grid(xs_blocks(g.n0 * g.n1, XL<T, N2>::LPW), nprob);
  k_x_stokes_local<T, N2><<<grid, XS_WARPS * 32, smem, s>>>((const cx<T>*)spec, (T*)u, (T*)lam, H, Hb, prm, part, g,
                                                            (const cx<T>*)tw);
  return cudaGetLastError();
}

template <typename T, int N2>
static cudaError_t l_x_rhs(const Geo& g, int nprob, void* spec, const void* u, const void* lam, const uint8_t* H,
                           const uint32_t* Hb, const StokesDev* prm, const void* tw, cudaStream_t s) {
  constexpr int smem = xs_smem_bytes<T, N2, 1, 0>();
  static const cudaError_t attr = set_smem(k_x_stokes_rhs<T, N2>, smem);
  if (attr != cudaSuccess) return attr;
  dim3 grid(xs_blocks(g.n0 * g.n1, XL<T, N2>::LPW), nprob);
  k_x_stokes_rhs<T, N2><<<grid, XS_WARPS * 32, smem, s>>>((cx<T>*)spec, (const T*)u, (const T*)lam, H, Hb, prm, g,
                                                          (const cx<T>*)tw);
  return cudaGetLastError();
}

template <typename T, int N2>
static cudaError_t l_x_solute(const Geo& g, int nprob, void* spec, const void* u, const uint8_t* H,
                              const uint32_t* Hb, const SoluteDev* prm, const void* tw, const T* d2, bool central,
                              cudaStream_t s) {
  constexpr int smem = xs_smem_bytes<T, N2, 2, 2 * XL<T, N2>::E>();
  static const cudaError_t attr0 = set_smem(k_x_solute<T, N2, false>, smem);
  static const cudaError_t attr1 = set_smem(k_x_solute<T, N2, true>, smem);
  if (attr0 != cudaSuccess) return attr0;
  if (attr1 != cudaSuccess) return attr1;
  // problems sharing the velocity and the indicator loop inside the kernel (up
  // to XS_PCACHE per block), with fewer line groups per warp so that the grid
  // keeps its size
  const bool shared = g.us == 0 && g.hs == 0;
  const int np_blk = nprob < XS_PCACHE ? nprob : XS_PCACHE;
  const int gpw = shared ? (XS_GPW / np_blk > 1 ? XS_GPW / np_blk : 1) : XS_GPW;
  const int ngroups = g.n0 * g.n1 / XL<T, N2>::LPW;
  dim3 grid((ngroups + XS_WARPS * gpw - 1) / (XS_WARPS * gpw), shared ? (nprob + XS_PCACHE - 1) / XS_PCACHE : nprob);
  if (central)
    k_x_solute<T, N2, true><<<grid, XS_WARPS * 32, smem, s>>>((cx<T>*)spec, (const T*)u, H, Hb, prm, g,
                                                               (const cx<T>*)tw, d2, nprob, gpw);
  else
    k_x_solute<T, N2, false><<<grid, XS_WARPS * 32, smem, s>>>((cx<T>*)spec, (const T*)u, H, Hb, prm, g,
                                                                (const cx<T>*)tw, d2, nprob, gpw);
  return cudaGetLastError();
}

template <typename T, int N2, int NC>
static cudaError_t l_x_r2c_nc(const Geo& g, int nprob, void* spec, long long sps, const void* in, long long ips,
                              const void* tw, cudaStream_t s) {
  constexpr int smem = x_smem_bytes<T, N2, NC>();
  static const cudaError_t attr = set_smem(k_x_r2c<T, N2, NC>, smem);
  if (attr != cudaSuccess) return attr;
  dim3 grid(g.n0 * g.n1 / XCfg<T, N2>::LPB, nprob);
  k_x_r2c<T, N2, NC><<<grid, NC * 64, smem, s>>>((cx<T>*)spec, (const T*)in, g, ips, sps, (const cx<T>*)tw);
  return cudaGetLastError();
}
template <typename T, int N2>
static cudaError_t l_x_r2c(const Geo& g, int nprob, int nc, void* spec, long long sps, const void* in,
                           long long ips, const void* tw, cudaStream_t s) {
  if (nc == 1) return l_x_r2c_nc<T, N2, 1>(g, nprob, spec, sps, in, ips, tw, s);
  if (nc == 3) return l_x_r2c_nc<T, N2, 3>(g, nprob, spec, sps, in, ips, tw, s);
  return cudaErrorInvalidValue;
}

template <typename T, int N2, int NC>
static cudaError_t l_x_c2r_nc(const Geo& g, int nprob, const void* spec, long long sps, void* out, long long ops,
                              const void* tw, cudaStream_t s) {
  constexpr int smem = x_smem_bytes<T, N2, NC>();
  static const cudaError_t attr = set_smem(k_x_c2r<T, N2, NC>, smem);
  if (attr != cudaSuccess) return attr;
  dim3 grid(g.n0 * g.n1 / XCfg<T, N2>::LPB, nprob);
  k_x_c2r<T, N2, NC><<<grid, NC * 64, smem, s>>>((const cx<T>*)spec, (T*)out, g, ops, sps, (const cx<T>*)tw);
  return cudaGetLastError();
}
// The line-resident kernel stores voxel pairs as vectors: it runs when `out`
// is aligned to a pair (the strides are even); otherwise the block-phase
// kernel with element stores does.
template <typename T, int N2>
static cudaError_t l_x_c2r(const Geo& g, int nprob, int nc, const void* spec, long long sps, void* out,
                           long long ops, const void* tw, cudaStream_t s) {
  if ((uintptr_t)out % (2 * sizeof(T)) == 0 && ops % 2 == 0 && g.V % 2 == 0) {
    constexpr int smem = xs_smem_bytes<T, N2, 1, 0>();
    static const cudaError_t attr = set_smem(k_x_c2r_lr<T, N2>, smem);
    if (attr != cudaSuccess) return attr;
    dim3 grid(xs_blocks(g.n0 * g.n1, XL<T, N2>::LPW), nprob * nc);
    k_x_c2r_lr<T, N2><<<grid, XS_WARPS * 32, smem, s>>>((const cx<T>*)spec, (T*)out, g, nc, ops, sps,
                                                        (const cx<T>*)tw);
    return cudaGetLastError();
  }
  if (nc == 1) return l_x_c2r_nc<T, N2, 1>(g, nprob, spec, sps, out, ops, tw, s);
  if (nc == 3) return l_x_c2r_nc<T, N2, 3>(g, nprob, spec, sps, out, ops, tw, s);
  return cudaErrorInvalidValue;
}

// Autotuner candidates: the passes of the solver loops at N >= 64 also exist
// with half, double and four times the default tile width, when the variant
// stays within 2..32 columns, 1536 line threads (run in rounds of at most 512
// or 1024) and 200 KB of shared memory. Wide tiles read longer row segments,
// which matters most along the slowest axis.
template <int N, int OP, int NC>
constexpr bool tunable() {
  return N >= 64 && ((OP == OP_FWD && NC == 3) || (OP == OP_INV && NC == 3) || OP == OP_STOKES || OP == OP_SOLUTE ||
                     OP == OP_FWD_SOL || OP == OP_INV_SOL);
}

template <typename T, int N, int OP, int NC, int TX>
constexpr bool tx_ok() {
  return TX >= 2 && TX <= 32 && NC * TX * (N / ept(N)) <= 1536 &&
         (NC * TX * line_stride(N, N / ept(N), TX, wave_slots<T>()) + tw_total(N)) * (int)sizeof(cx<T>) <= 200 * 1024;
}

// The register-resident variant (acm_rpass.cuh) of a tunable pass: lines of
// 64, 128 or 256 points.
template <typename T, int N, int OP, int NC>
constexpr bool rr_ok() {
  return (N == 64 || N == 128 || N == 256) && tunable<N, OP, NC>();
}

// tile width of (T, N, OP, NC) under the choice `shift`; the register-resident
// variants (shift 3: W = rr_wdef, shift 4: W = rr_wdef / 2 columns per block)
// report -W
template <typename T, int N, int OP, int NC>
constexpr int resolved_tx(int shift) {
  constexpr int TX0 = pick_tx((int)sizeof(cx<T>), N, NC);
  if constexpr (rr_ok<T, N, OP, NC>()) {
    if (shift == 3) return -rr_wdef<T>();
    if (shift == 4) return -rr_wdef<T>() / 2;
  }
  if (tunable<N, OP, NC>()) {
    if (shift < 0 && tx_ok<T, N, OP, NC, TX0 / 2>()) return TX0 / 2;
    if (shift == 1 && tx_ok<T, N, OP, NC, TX0 * 2>()) return TX0 * 2;
    if (shift == 2 && tx_ok<T, N, OP, NC, TX0 * 4>()) return TX0 * 4;
  }
  return TX0;
}

template <typename T>
static PassArgs<T> pass_args(const Geo& g, int axis, void* spec, long long probStride, const Sym<T>& sym,
                             const void* tw, void* st0, void* st1, StokesDev* sprm, SoluteDev* cprm, double* part,
                             int dm) {
  PassArgs<T> a;
  a.spec = (cx<T>*)spec;
  a.probStride = probStride;
  a.compStride = g.S;
  if (axis == 1) {
    a.rowStride = g.P;
    a.outerStride = (long long)g.n1 * g.P;
  } else {
    a.rowStride = (long long)g.n1 * g.P;
    a.outerStride = g.P;
  }
  a.Pu = g.Pu;
  a.n1 = g.n1;
  a.sym = sym;
  a.twg = (const cx<T>*)tw;
  a.st0 = (cx<T>*)st0;
  a.st1 = (cx<T>*)st1;
  a.sprm = sprm;
  a.cprm = cprm;
  a.part = part;
  a.invV = 1.0 / (double)g.V;
  a.nkx = g.n2 / 2;
  a.dm = dm;
  a.nouter = axis == 1 ? g.n0 : g.n1;
  return a;
}

template <typename T, int N, int OP, int NC, int TX>
static cudaError_t l_pass_kt(const Geo& g, int axis, int nprob, void* spec, long long probStride, const Sym<T>& sym,
                             const void* tw, void* st0, void* st1, StokesDev* sprm, SoluteDev* cprm, double* part,
                             cudaStream_t s, int dm) {
  using C = SCfg<T, N, OP, NC, TX>;
  static const cudaError_t attr = set_smem(k_strided<T, N, OP, NC, TX>, C::SMEM);
  if (attr != cudaSuccess) return attr;
  const PassArgs<T> a = pass_args<T>(g, axis, spec, probStride, sym, tw, st0, st1, sprm, cprm, part, dm);
  const int nouter = axis == 1 ? g.n0 : g.n1;
  dim3 grid((g.Pu + TX - 1) / TX, nouter, nprob);
  k_strided<T, N, OP, NC, TX><<<grid, C::NT, C::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int N, int OP, int NC, int W>
static cudaError_t l_pass_rr(const Geo& g, int axis, int nprob, void* spec, long long probStride, const Sym<T>& sym,
                             const void* tw, void* st0, void* st1, StokesDev* sprm, SoluteDev* cprm, double* part,
                             cudaStream_t s) {
  using C = RCfg<T, N, W>;
  constexpr int smem = rr_smem<T, N, OP, NC, W>();
  constexpr bool wide = rr_y_wide<T, OP, W>() && N == 256;
  static const cudaError_t attr = [] {
    if constexpr (wide) return set_smem(k_rstrided_w<T, N, OP, NC, W>, smem);
    else return set_smem(k_rstrided<T, N, OP, NC, W>, smem);
  }();
  if (attr != cudaSuccess) return attr;
  const PassArgs<T> a = pass_args<T>(g, axis, spec, probStride, sym, tw, st0, st1, sprm, cprm, part, 0);
  const RTiles tl = rr_tiles(g.Pu, a.nouter, W);
  if constexpr (wide) k_rstrided_w<T, N, OP, NC, W><<<nprob * tl.nlive, C::NT, smem, s>>>(a);
  else k_rstrided<T, N, OP, NC, W><<<nprob * tl.nlive, C::NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int N, int OP, int NC>
static cudaError_t l_pass_k(const Geo& g, int axis, int nprob, void* spec, long long probStride, const Sym<T>& sym,
                            const void* tw, void* st0, void* st1, StokesDev* sprm, SoluteDev* cprm, double* part,
                            cudaStream_t s, int dm) {
  constexpr int TX0 = pick_tx((int)sizeof(cx<T>), N, NC);
  if constexpr (rr_ok<T, N, OP, NC>()) {
    const int sh = g.txs[sizeof(T) == 8][axis][OP];
    if (sh == 3)
      return l_pass_rr<T, N, OP, NC, rr_wdef<T>()>(g, axis, nprob, spec, probStride, sym, tw, st0, st1, sprm, cprm,
                                                   part, s);
    if (sh == 4)
      return l_pass_rr<T, N, OP, NC, rr_wdef<T>() / 2>(g, axis, nprob, spec, probStride, sym, tw, st0, st1, sprm,
                                                       cprm, part, s);
  }
  if constexpr (tunable<N, OP, NC>()) {
    const int sh = g.txs[sizeof(T) == 8][axis][OP];
    if constexpr (tx_ok<T, N, OP, NC, TX0 / 2>())
      if (sh < 0)
        return l_pass_kt<T, N, OP, NC, TX0 / 2>(g, axis, nprob, spec, probStride, sym, tw, st0, st1, sprm, cprm,
                                                part, s, dm);
    if constexpr (tx_ok<T, N, OP, NC, TX0 * 2>())
      if (sh == 1)
        return l_pass_kt<T, N, OP, NC, TX0 * 2>(g, axis, nprob, spec, probStride, sym, tw, st0, st1, sprm, cprm,
                                                part, s, dm);
    if constexpr (tx_ok<T, N, OP, NC, TX0 * 4>())
      if (sh == 2)
        return l_pass_kt<T, N, OP, NC, TX0 * 4>(g, axis, nprob, spec, probStride, sym, tw, st0, st1, sprm, cprm,
                                                part, s, dm);
  }
  return l_pass_kt<T, N, OP, NC, TX0>(g, axis, nprob, spec, probStride, sym, tw, st0, st1, sprm, cprm, part, s, dm);
}

template <typename T, int N>
static int l_pass_tx(int op, int nc, int shift) {
#define ACM_TX(OPV, NCV) \
  if (op == OPV && nc == NCV) return resolved_tx<T, N, OPV, NCV>(shift);
  ACM_TX(OP_FWD, 1)
  ACM_TX(OP_FWD, 3)
  ACM_TX(OP_FWD, 4)
  ACM_TX(OP_INV, 1)
  ACM_TX(OP_INV, 3)
  ACM_TX(OP_INV_SCALE, 1)
  ACM_TX(OP_STOKES, 3)
  ACM_TX(OP_SOLUTE, 2)
  ACM_TX(OP_FWD_SOL, 3)
  ACM_TX(OP_INV_SOL, 3)
  ACM_TX(OP_DERIV, 1)
#undef ACM_TX
  return 0;
}

template <typename T, int N>
static cudaError_t l_pass(const Geo& g, int axis, int op, int nc, int nprob, void* spec, long long ps,
                          const Sym<T>& sym, const void* tw, void* st0, void* st1, StokesDev* sprm, SoluteDev* cprm,
                          double* part, cudaStream_t s, int dm) {
#define ACM_PASS(OPV, NCV)                                                                                    \
  if (op == OPV && nc == NCV)                                                                                 \
    return l_pass_k<T, N, OPV, NCV>(g, axis, nprob, spec, ps, sym, tw, st0, st1, sprm, cprm, part, s, dm);
  ACM_PASS(OP_FWD, 1)
  ACM_PASS(OP_FWD, 3)
  ACM_PASS(OP_FWD, 4)
  ACM_PASS(OP_INV, 1)
  ACM_PASS(OP_INV, 3)
  ACM_PASS(OP_INV_SCALE, 1)
  ACM_PASS(OP_STOKES, 3)
  ACM_PASS(OP_SOLUTE, 2)
  ACM_PASS(OP_FWD_SOL, 3)
  ACM_PASS(OP_INV_SOL, 3)
  ACM_PASS(OP_DERIV, 1)
#undef ACM_PASS
  return cudaErrorInvalidValue;
}

template <typename T>
int Ops<T>::x_blocks(const Geo& g) {
  const int M = g.n2 / 2;
  const int TL = M / ept(M);
  return xs_blocks(g.n0 * g.n1, 32 / TL);
}

template <typename T>
int Ops<T>::pass_tx(const Geo& g, int axis, int op, int nc) {
  const int n = axis == 1 ? g.n1 : g.n0;
  const int sh = g.txs[sizeof(T) == 8][axis][op];
  switch (n) {
    case 1: return l_pass_tx<T, 1>(op, nc, sh);
    case 8: return l_pass_tx<T, 8>(op, nc, sh);
    case 16: return l_pass_tx<T, 16>(op, nc, sh);
    case 32: return l_pass_tx<T, 32>(op, nc, sh);
    case 64: return l_pass_tx<T, 64>(op, nc, sh);
    case 128: return l_pass_tx<T, 128>(op, nc, sh);
    case 256: return l_pass_tx<T, 256>(op, nc, sh);
    case 512: return l_pass_tx<T, 512>(op, nc, sh);
    default: return 0;
  }
}

template <typename T>
bool Ops<T>::tx_variant(int n, int op, int nc, int shift) {
  Geo g;
  g.n0 = g.n1 = n;
  const int t0 = pass_tx(g, 0, op, nc);
  g.txs[sizeof(T) == 8][0][op] = (signed char)shift;
  const int t1 = pass_tx(g, 0, op, nc);
  if (shift >= 3) return t1 < 0;
  return shift == 0 || (t1 != t0 && t1 > 0);
}

template <typename T>
int Ops<T>::z_blocks(const Geo& g, int op) {
  const int nc = op == P_SOLUTE ? 2 : 3;
  const int tx = pass_tx(g, 0, op, nc);
  if (tx < 0) return rr_tiles(g.Pu, g.n1, -tx).nlive;   // register-resident: one record per live tile
  return ((g.Pu + tx - 1) / tx) * g.n1;
}

template <typename T>
cudaError_t Ops<T>::x_stokes_local(const Geo& g, int nprob, const void* spec, void* u, void* lam, const uint8_t* H,
                                   const uint32_t* Hb, StokesDev* prm, double* part, const void* tw, cudaStream_t s) {
  ACM_DISPATCH_N(g.n2, l_x_local, g, nprob, spec, u, lam, H, Hb, prm, part, tw, s)
}

template <typename T>
cudaError_t Ops<T>::x_stokes_rhs(const Geo& g, int nprob, void* spec, const void* u, const void* lam,
                                 const uint8_t* H, const uint32_t* Hb, const StokesDev* prm, const void* tw,
                                 cudaStream_t s) {
  ACM_DISPATCH_N(g.n2, l_x_rhs, g, nprob, spec, u, lam, H, Hb, prm, tw, s)
}

template <typename T>
cudaError_t Ops<T>::x_solute(const Geo& g, int nprob, void* spec, const void* u, const uint8_t* H,
                             const uint32_t* Hb, const SoluteDev* prm, const void* tw, const Sym<T>& sym,
                             bool central, cudaStream_t s) {
  ACM_DISPATCH_N(g.n2, l_x_solute, g, nprob, spec, u, H, Hb, prm, tw, sym.d2, central, s)
}

template <typename T>
cudaError_t Ops<T>::x_r2c(const Geo& g, int nprob, int nc, void* spec, long long sps, const void* in, long long ips,
                          const void* tw, cudaStream_t s) {
  ACM_DISPATCH_N(g.n2, l_x_r2c, g, nprob, nc, spec, sps, in, ips, tw, s)
}

template <typename T>
cudaError_t Ops<T>::x_c2r(const Geo& g, int nprob, int nc, const void* spec, long long sps, void* out,
                          long long ops, const void* tw, cudaStream_t s) {
  ACM_DISPATCH_N(g.n2, l_x_c2r, g, nprob, nc, spec, sps, out, ops, tw, s)
}

template <typename T>
cudaError_t Ops<T>::pass(const Geo& g, int axis, int op, int nc, int nprob, void* spec, long long ps,
                         const Sym<T>& sym, const void* tw, void* st0, void* st1, StokesDev* sprm, SoluteDev* cprm,
                         double* part, cudaStream_t s, int dm) {
  const int n = axis == 1 ? g.n1 : g.n0;
  if ((op == P_STOKES || op == P_SOLUTE || op == P_DERIV) && axis != 0) return cudaErrorInvalidValue;
  if ((op == P_FWD_SOL || op == P_INV_SOL) && axis != 1) return cudaErrorInvalidValue;
  ACM_DISPATCH_NS(n, l_pass, g, axis, op, nc, nprob, spec, ps, sym, tw, st0, st1, sprm, cprm, part, s, dm)
}

template <typename T>
cudaError_t Ops<T>::pore_products(const Geo& g, const void* f, const uint8_t* H, double* part, int nblk,
                                  cudaStream_t s) {
  k_pore_products<T><<<nblk, 256, 0, s>>>((const T*)f, H, g.V, part);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::field_sums(const Geo& g, int nprob, const void* u, const uint8_t* H, double* part, int nblk,
                               cudaStream_t s) {
  dim3 grid(nblk, nprob);
  k_field_sums<T><<<grid, 256, 0, s>>>((const T*)u, H, g.V, g.us, g.hs, part);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::diffusivity(const Geo& g, int nprob, const void* chi, const void* grad, const void* u,
                                const uint8_t* H, const SoluteDev* prm, double* part, int nblk, cudaStream_t s) {
  dim3 grid(nblk, nprob);
  k_diffusivity<T><<<grid, 256, 0, s>>>((const T*)chi, (const T*)grad, (const T*)u, H, g.V, g.us, g.hs, prm, part);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::mask_solid(const Geo& g, const void* in, void* out, const uint8_t* H, cudaStream_t s) {
  k_mask_solid<T><<<608, 256, 0, s>>>((const T*)in, (T*)out, H, g.V);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::div_spec(const Geo& g, const void* uh, void* dv, const Sym<T>& sym, cudaStream_t s) {
  k_div_spec<T><<<608, 256, 0, s>>>((const cx<T>*)uh, (cx<T>*)dv, g, sym);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::q_from_a(const Geo& g, const void* ah, void* q, const Sym<T>& sym, cudaStream_t s) {
  k_q_from_a<T><<<608, 256, 0, s>>>((const cx<T>*)ah, (cx<T>*)q, g, sym);
  return cudaGetLastError();
}

}  // namespace acm
