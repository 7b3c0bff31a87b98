// acm_api.cu -- the C ABI (include/acm.h): contexts, workspace, and the
// device-resident iteration drivers of Algorithm 1 (Problems 1 and 2).
//
// Each solve runs entirely on the context's stream. The host only launches
// kernels and, every `check_every` iterations, reads the per-problem stop flags
// that the FP64 finalize kernel writes (no per-iteration synchronisation).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "acm.h"
#include "acm_ops.h"

using namespace acm;

namespace {

constexpr int BMAX = 3;          // problems of the single-cell entry points (three loads)
constexpr int HIST_CAP = 20000;  // per-problem history records
constexpr int NRED = 304;        // blocks of the FP64 field reductions
// iterations without a 2 % gain towards the tolerance after which the FP32
// phase of ACM_FP32_THEN_FP64 hands a problem over to FP64
constexpr int STALL_WINDOW = 500;

struct Prec {
  bool ready = false;
  void* spec = nullptr;  // [BMAX][4][S] complex
  void* st0 = nullptr;   // [BMAX][S] complex: q^ (Stokes) or chi^ (solute)
  void* st1 = nullptr;   // [BMAX][S] complex: div^ of the previous iteration
  void* u = nullptr;     // [BMAX][3][V] real
  void* lam = nullptr;   // [BMAX][3][V] real: H lambda
  void* aux = nullptr;   // [B][4][V] real, allocated on first use: staging, grad chi [B][3][V], chi [B][V]
  void* tw = nullptr;    // [TW_MAX] complex twiddles W_1024^k
  void* sym = nullptr;   // two symbol sets (EXACT, CENTRAL)
};

template <typename T>
struct CxT {
  T x, y;
};

}  // namespace

// What a captured loop depends on beyond its buffers: precision, problems,
// derivative symbols, kind (1 Stokes, 2 solute), iteration cap and the caller
// buffers it reads in place (the solute's velocity and indicator).
struct GraphKey {
  int prec = -1, nprob = -1, deriv = -1, kind = -1;
  unsigned cap = 0;
  const void* kp = nullptr;
  const void* kq = nullptr;
  long long kx = 0;
  bool operator==(const GraphKey& o) const {
    return prec == o.prec && nprob == o.nprob && deriv == o.deriv && kind == o.kind && cap == o.cap &&
           kp == o.kp && kq == o.kq && kx == o.kx;
  }
};

struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  GraphKey key;
  unsigned int* counter = nullptr;  // device iteration counter of the loop
};

struct acm_ctx {
  int n0, n1, n2;
  Geo g;
  cudaStream_t st;
  int B = BMAX;       // problem capacity of the workspace
  int ncells = 1;     // indicator slots in Hd (cells of a batch)
  int spec_comps = 4; // spectral components per problem (3 suffice for Stokes-only batches)
  GraphCache graph;      // the Stokes loop
  GraphCache graph_sol;  // the solute loop
  cudaStream_t cap = nullptr;  // non-blocking stream used only to capture graphs
  Prec pf, pd;
  StokesDev* sprm = nullptr;
  SoluteDev* cprm = nullptr;
  double* part_x = nullptr;
  double* part_z = nullptr;
  double* part_r = nullptr;
  int nbx = 0, nbz = 0;
  uint8_t* Hd = nullptr;
  uint32_t* Hb = nullptr;   // [ncells][V / 32] indicator bits (x passes)
  unsigned long long* cnt = nullptr;
  double* hist = nullptr;
  int solute_deriv = 1;      // derivative symbol of the last solute iteration
  double* hist_b = nullptr;  // batches: [B][hist_b_cap][STOKES_HIST] when enabled
  int hist_b_cap = 0;
  int hist_kind = 0;  // 1: Stokes (16 doubles / record), 2: solute (4 doubles / record)
  int hist_n[BMAX] = {0, 0, 0};
  void* pin = nullptr;  // pinned host scratch
  size_t pin_bytes = 0;
  // profiler
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
  std::vector<std::pair<int, size_t>> recs;  // (kind, index of the start event)
  long long launches[ACM_K_COUNT] = {};
};

namespace {

thread_local char g_last_error[512] = "";

void note_error(cudaError_t e, const char* what, int line) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s (%s) at acm_api.cu:%d: %s", cudaGetErrorName(e),
                cudaGetErrorString(e), line, what);
}

#define CK(x)                               \
  do {                                      \
    cudaError_t e_ = (x);                   \
    if (e_ != cudaSuccess) {                \
      note_error(e_, #x, __LINE__);         \
      cudaGetLastError();                   \
      return ACM_ERR_CUDA;                  \
    }                                       \
  } while (0)

#define CKS(x)                              \
  do {                                      \
    acm_status s_ = (x);                    \
    if (s_ != ACM_OK) return s_;            \
  } while (0)

void prof_begin(acm_ctx* c, int kind) {
  c->launches[kind] += 1;
  if (!c->prof) return;
  while (c->ev.size() < c->ev_used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      c->prof = false;
      return;
    }
    c->ev.push_back(e);
  }
  cudaEventRecord(c->ev[c->ev_used], c->st);
  c->recs.push_back({kind, c->ev_used});
  c->ev_used += 2;
}

void prof_end(acm_ctx* c) {
  if (!c->prof || c->recs.empty()) return;
  cudaEventRecord(c->ev[c->recs.back().second + 1], c->st);
}

// launch through the profiler: one kernel launch of the given kind
#define LK(kind, x)                         \
  do {                                      \
    prof_begin(c, kind);                    \
    cudaError_t e_ = (x);                   \
    prof_end(c);                            \
    if (e_ != cudaSuccess) {                \
      note_error(e_, #x, __LINE__);         \
      cudaGetLastError();                   \
      return ACM_ERR_CUDA;                  \
    }                                       \
  } while (0)

bool pow2_in_range(int n) { return n >= 8 && n <= 512 && (n & (n - 1)) == 0; }

// Supported grids: n1, n2 powers of two in [8, 512]; n0 the same or 1 (a
// single plane: the two-dimensional problem of the paper's experiments).
// A plane cell needs n1 >= 32: the line-resident x passes hand lines out in
// groups of up to 32 (one warp), and a plane of fewer lines forms none.
bool shape_ok(int n0, int n1, int n2) {
  return (pow2_in_range(n0) || (n0 == 1 && n1 >= 32)) && pow2_in_range(n1) && pow2_in_range(n2);
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// captured loops hold kernel arguments (tile widths, buffers): drop them
// whenever those change
void drop_graphs(acm_ctx* c) {
  for (GraphCache* g : {&c->graph, &c->graph_sol}) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
  }
}

template <typename T>
Prec& prec(acm_ctx* c);
template <>
Prec& prec<float>(acm_ctx* c) { return c->pf; }
template <>
Prec& prec<double>(acm_ctx* c) { return c->pd; }

// per-axis symbols (Eq. 13 exact, Eq. 21 central); index m in FFT order
void axis_symbols(int n, int len, int deriv, std::vector<double>& d, std::vector<double>& l) {
  d.resize(len);
  l.resize(len);
  const double PI = 3.14159265358979323846;
  for (int m = 0; m < len; ++m) {
    const int ms = (m <= n / 2) ? m : m - n;
    const double k = 2.0 * PI * ms;
    if (deriv == ACM_DERIV_EXACT) {
      d[m] = (2 * m == n) ? 0.0 : k;
      l[m] = k * k;
    } else {
      d[m] = (2 * m == n || m == 0) ? 0.0 : std::sin(2.0 * PI * ms / n) * n;
      const double s = std::sin(PI * ms / n);
      l[m] = 4.0 * s * s * (double)n * n;
    }
  }
}

template <typename T>
size_t sym_count(const Geo& g) {
  return (size_t)2 * (g.n0 + g.n1 + g.Pu);
}

template <typename T>
Sym<T> sym_of(acm_ctx* c, int deriv) {
  const Geo& g = c->g;
  const T* base = (const T*)prec<T>(c).sym + (size_t)deriv * sym_count<T>(g);
  Sym<T> s;
  s.d0 = base;
  s.l0 = base + g.n0;
  s.d1 = base + 2 * g.n0;
  s.l1 = base + 2 * g.n0 + g.n1;
  s.d2 = base + 2 * (g.n0 + g.n1);
  s.l2 = base + 2 * (g.n0 + g.n1) + g.Pu;
  return s;
}

template <typename T>
acm_status ensure_prec(acm_ctx* c) {
  Prec& w = prec<T>(c);
  if (w.ready) return ACM_OK;
  const Geo& g = c->g;
  const size_t cs = 2 * sizeof(T);
  auto alloc = [&](void** p, size_t bytes) -> bool { return cudaMalloc(p, bytes) == cudaSuccess; };
  if (!alloc(&w.spec, (size_t)c->B * c->spec_comps * g.S * cs) || !alloc(&w.st0, (size_t)c->B * g.S * cs) ||
      !alloc(&w.st1, (size_t)c->B * g.S * cs) || !alloc(&w.u, (size_t)c->B * 3 * g.V * sizeof(T)) ||
      !alloc(&w.lam, (size_t)c->B * 3 * g.V * sizeof(T)) || !alloc(&w.tw, (size_t)TW_MAX * cs) ||
      !alloc(&w.sym, 2 * sym_count<T>(g) * sizeof(T))) {
    cudaGetLastError();
    return ACM_ERR_NOMEM;
  }
  // zero the spectral padding columns once (they are never written by the passes)
  CK(cudaMemset(w.spec, 0, (size_t)c->B * c->spec_comps * g.S * cs));
  CK(cudaMemset(w.st0, 0, (size_t)c->B * g.S * cs));
  CK(cudaMemset(w.st1, 0, (size_t)c->B * g.S * cs));
  std::vector<T> tw(2 * TW_MAX);
  const double PI = 3.14159265358979323846;
  for (int k = 0; k < TW_MAX; ++k) {
    tw[2 * k] = (T)std::cos(2.0 * PI * k / TW_MAX);
    tw[2 * k + 1] = (T)(-std::sin(2.0 * PI * k / TW_MAX));
  }
  CK(cudaMemcpy(w.tw, tw.data(), tw.size() * sizeof(T), cudaMemcpyHostToDevice));
  std::vector<T> sym;
  for (int deriv = 0; deriv < 2; ++deriv) {
    std::vector<double> d, l;
    axis_symbols(g.n0, g.n0, deriv, d, l);
    for (double x : d) sym.push_back((T)x);
    for (double x : l) sym.push_back((T)x);
    axis_symbols(g.n1, g.n1, deriv, d, l);
    for (double x : d) sym.push_back((T)x);
    for (double x : l) sym.push_back((T)x);
    axis_symbols(g.n2, g.Pu, deriv, d, l);
    for (double x : d) sym.push_back((T)x);
    for (double x : l) sym.push_back((T)x);
  }
  CK(cudaMemcpy(w.sym, sym.data(), sym.size() * sizeof(T), cudaMemcpyHostToDevice));
  w.ready = true;
  return ACM_OK;
}

// the auxiliary real buffer (staging of host inputs, solute and pressure outputs)
template <typename T>
acm_status ensure_aux(acm_ctx* c) {
  CKS(ensure_prec<T>(c));
  Prec& w = prec<T>(c);
  if (w.aux) return ACM_OK;
  if (cudaMalloc(&w.aux, (size_t)c->B * 4 * c->g.V * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    w.aux = nullptr;
    return ACM_ERR_NOMEM;
  }
  return ACM_OK;
}

void free_prec(Prec& w) {
  void* ps[] = {w.spec, w.st0, w.st1, w.u, w.lam, w.aux, w.tw, w.sym};
  for (void* p : ps)
    if (p) cudaFree(p);
  w = Prec();
}

acm_status pin_scratch(acm_ctx* c, size_t bytes) {
  if (c->pin_bytes >= bytes) return ACM_OK;
  if (c->pin) cudaFreeHost(c->pin);
  c->pin = nullptr;
  c->pin_bytes = 0;
  if (cudaMallocHost(&c->pin, bytes) != cudaSuccess) {
    cudaGetLastError();
    return ACM_ERR_NOMEM;
  }
  c->pin_bytes = bytes;
  return ACM_OK;
}

// H to device memory (staged when it is a host buffer); counts solid voxels
acm_status stage_H(acm_ctx* c, const uint8_t* H, const uint8_t** Hdev, long long* nsolid) {
  const Geo& g = c->g;
  // the kernels stage H with 16-byte asynchronous copies: use a device buffer in
  // place only when it is 16-byte aligned
  if (is_device_ptr(H) && ((uintptr_t)H & 15) == 0) {
    *Hdev = H;
  } else {
    CK(cudaMemcpyAsync(c->Hd, H, (size_t)g.V, cudaMemcpyDefault, c->st));
    *Hdev = c->Hd;
  }
  LK(ACM_K_OTHER, count_solid(*Hdev, g.V, c->cnt, c->st));
  CKS(pin_scratch(c, 1 << 20));
  CK(cudaMemcpyAsync(c->pin, c->cnt, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  *nsolid = (long long)*(unsigned long long*)c->pin;
  return ACM_OK;
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// sum of NRED FP64 partial records (stride 8) per problem, in a fixed order
acm_status read_partials(acm_ctx* c, int nprob, int nval, std::vector<double>& out) {
  CKS(pin_scratch(c, (size_t)nprob * NRED * 8 * sizeof(double)));
  CK(cudaMemcpyAsync(c->pin, c->part_r, (size_t)nprob * NRED * 8 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  const double* h = (const double*)c->pin;
  out.assign((size_t)nprob * nval, 0.0);
  for (int p = 0; p < nprob; ++p)
    for (int i = 0; i < NRED; ++i)
      for (int k = 0; k < nval; ++k) out[(size_t)p * nval + k] += h[((size_t)p * NRED + i) * 8 + k];
  return ACM_OK;
}

// ---------------------------------------------------------------------------
// Stokes (Section 3.1, Algorithm 1 Problem 1)
// ---------------------------------------------------------------------------
struct StokesCfg {
  acm_stokes_params prm;
  double psi0[3];
};

void fill_stokes_params(const acm_stokes_params* in, acm_stokes_params* out) {
  acm_stokes_default_params(out);
  if (in) *out = *in;
}

double default_penalty(const Geo& g, double nu) {
  // nu times the squared wavenumber of the geometric-mean grid spacing / 8, the
  // mean taken over the axes longer than one voxel (both in-plane axes of a plane)
  const double n = g.n0 > 1 ? std::cbrt((double)g.n0 * g.n1 * g.n2) : std::sqrt((double)g.n1 * g.n2);
  const double PI = 3.14159265358979323846;
  return nu * (PI * n) * (PI * n) / 8.0;
}

template <typename T>
acm_status stokes_setup(acm_ctx* c, int nprob, const uint8_t* Hdev, long long hs, int lph, const double (*gs)[3],
                        const acm_stokes_params& P, double eps, const void* const* init_u,
                        const void* const* init_lam, const int* preset_status = nullptr, int stall_win = 0,
                        const double* pore_l = nullptr) {
  CKS(ensure_prec<T>(c));
  Prec& w = prec<T>(c);
  Geo g = c->g;
  g.hs = hs;
  g.lph = lph;
  const size_t cs = 2 * sizeof(T);
  CK(cudaMemsetAsync(w.u, 0, (size_t)nprob * 3 * g.V * sizeof(T), c->st));
  CK(cudaMemsetAsync(w.lam, 0, (size_t)nprob * 3 * g.V * sizeof(T), c->st));
  CK(cudaMemsetAsync(w.st0, 0, (size_t)nprob * g.S * cs, c->st));
  CK(cudaMemsetAsync(w.st1, 0, (size_t)nprob * g.S * cs, c->st));
  const Sym<T> sym = sym_of<T>(c, P.deriv);
  for (int p = 0; p < nprob; ++p) {
    T* up = (T*)w.u + (size_t)p * 3 * g.V;
    T* lp = (T*)w.lam + (size_t)p * 3 * g.V;
    if (init_u && init_u[p]) {
      CK(cudaMemcpyAsync(up, init_u[p], 3 * g.V * sizeof(T), cudaMemcpyDefault, c->st));
      // div u^0 in Fourier space for the first dual residual of pair 2
      void* sp = (char*)w.spec;
      LK(ACM_K_OTHER, Ops<T>::x_r2c(g, 1, 3, sp, 3 * g.S, up, 3 * g.V, w.tw, c->st));
      LK(ACM_K_OTHER, Ops<T>::pass(g, 1, P_FWD, 3, 1, sp, 3 * g.S, sym, w.tw, nullptr, nullptr, nullptr, nullptr, nullptr, c->st));
      LK(ACM_K_OTHER, Ops<T>::pass(g, 0, P_FWD, 3, 1, sp, 3 * g.S, sym, w.tw, nullptr, nullptr, nullptr, nullptr, nullptr, c->st));
      LK(ACM_K_OTHER, Ops<T>::div_spec(g, sp, (char*)w.st1 + (size_t)p * g.S * cs, sym, c->st));
    }
    if (init_lam && init_lam[p]) {
      CKS(ensure_aux<T>(c));
      CK(cudaMemcpyAsync(w.aux, init_lam[p], 3 * g.V * sizeof(T), cudaMemcpyDefault, c->st));
      LK(ACM_K_OTHER, Ops<T>::mask_solid(g, w.aux, lp, Hdev + (size_t)(p / lph) * hs, c->st));
      // q^0: the pressure consistent with a^0 = H lambda^0 at a fixed point
      void* sp = (char*)w.spec;
      LK(ACM_K_OTHER, Ops<T>::x_r2c(g, 1, 3, sp, 3 * g.S, lp, 3 * g.V, w.tw, c->st));
      LK(ACM_K_OTHER, Ops<T>::pass(g, 1, P_FWD, 3, 1, sp, 3 * g.S, sym, w.tw, nullptr, nullptr, nullptr, nullptr, nullptr, c->st));
      LK(ACM_K_OTHER, Ops<T>::pass(g, 0, P_FWD, 3, 1, sp, 3 * g.S, sym, w.tw, nullptr, nullptr, nullptr, nullptr, nullptr, c->st));
      LK(ACM_K_OTHER, Ops<T>::q_from_a(g, sp, (char*)w.st0 + (size_t)p * g.S * cs, sym, c->st));
    }
  }
  std::vector<StokesDev> hp(nprob);
  const double p0 = default_penalty(g, P.nu);
  for (int p = 0; p < nprob; ++p) {
    StokesDev& d = hp[p];
    std::memset(&d, 0, sizeof(d));
    d.nu = P.nu;
    d.eps = eps;
    for (int k = 0; k < 3; ++k) {
      d.g[k] = gs[p][k];
      d.phi[k] = P.phi[k];
      d.tau[k] = P.tau[k];
    }
    // pore-scale rule: penalties not given start at pore_scale / l^2 times the default
    const double pd = (P.pore_scale > 0 && pore_l && pore_l[p] > 0) ? p0 * P.pore_scale / (pore_l[p] * pore_l[p]) : p0;
    d.psi[0] = P.alpha0 > 0 ? P.alpha0 : pd;
    d.psi[1] = P.beta0 > 0 ? P.beta0 : pd;
    d.psi[2] = P.b0 > 0 ? P.b0 : pd;
    for (int k = 0; k < 3; ++k) d.psi_min[k] = P.psi_min_frac * d.psi[k];
    // u~^0 = u^0 on the solid: s_prev = b_prev / (b_prev + alpha_prev) = 1
    d.psi_prev[0] = 0.0;
    d.psi_prev[1] = d.psi[1];
    d.psi_prev[2] = 1.0;
    for (int k = 0; k < 3; ++k) d.psi_last[k] = d.psi[k];
    d.adaptive = P.adaptive;
    d.max_iter = P.max_iter;
    d.stall_win = stall_win;
    d.stall_best = 1e300;
    if (preset_status && preset_status[p] != ACM_OK) {  // degenerate cell: not iterated
      d.done = 1;
      d.status = preset_status[p];
    }
  }
  CK(cudaMemcpyAsync(c->sprm, hp.data(), nprob * sizeof(StokesDev), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  return ACM_OK;
}

// step 1 of the coming iteration (Eq. 7 / Eq. 13): w -> u^ -> u (up to the x-pass)
template <typename T>
acm_status stokes_step1(acm_ctx* c, int nprob, const uint8_t* Hdev, long long hs, int lph, const Sym<T>& sym) {
  Prec& w = prec<T>(c);
  Geo g = c->g;
  g.hs = hs;
  g.lph = lph;
  const long long ps = 3 * g.S;
  LK(ACM_K_X_STOKES_RHS, Ops<T>::x_stokes_rhs(g, nprob, w.spec, w.u, w.lam, Hdev, c->Hb, c->sprm, w.tw, c->st));
  LK(ACM_K_Y_FWD_STOKES, Ops<T>::pass(g, 1, P_FWD, 3, nprob, w.spec, ps, sym, w.tw, nullptr, nullptr, c->sprm, nullptr, nullptr, c->st));
  LK(ACM_K_Z_STOKES, Ops<T>::pass(g, 0, P_STOKES, 3, nprob, w.spec, ps, sym, w.tw, w.st0, w.st1, c->sprm, nullptr, c->part_z, c->st));
  LK(ACM_K_Y_INV_STOKES, Ops<T>::pass(g, 1, P_INV, 3, nprob, w.spec, ps, sym, w.tw, nullptr, nullptr, c->sprm, nullptr, nullptr, c->st));
  return ACM_OK;
}

// One ADMM iteration of nprob problems after the previous one's step 1:
// steps 2-4 (x pass + finalize), then step 1 of the next iteration.
template <typename T>
acm_status stokes_body(acm_ctx* c, int nprob, const uint8_t* Hdev, long long hs, int lph, const Sym<T>& sym,
                       bool last) {
  Prec& w = prec<T>(c);
  Geo g = c->g;
  g.hs = hs;
  g.lph = lph;
  const int nbx = Ops<T>::x_blocks(g), nbz = Ops<T>::z_blocks(g, P_STOKES);
  double* hist = c->hist_b ? c->hist_b : (nprob <= BMAX ? c->hist : nullptr);
  const int hcap = c->hist_b ? c->hist_b_cap : HIST_CAP;
  LK(ACM_K_X_STOKES_LOCAL, Ops<T>::x_stokes_local(g, nprob, w.spec, w.u, w.lam, Hdev, c->Hb, c->sprm, c->part_x, w.tw,
                                                  c->st));
  LK(ACM_K_FINALIZE, stokes_finalize(nprob, c->sprm, c->part_x, nbx, c->part_z, nbz, (double)g.V, hist, hcap, c->st));
  if (!last) CKS(stokes_step1<T>(c, nprob, Hdev, hs, lph, sym));
  return ACM_OK;
}

struct StokesGroup {
  acm_ctx* c;
  int nprob;
  const uint8_t* H;
  long long hs;
  int lph;
};

// Device-resident loop: a CUDA graph whose while node repeats the work that
// `capture` enqueues (one iteration of every context in `ctxs`) followed by
// the loop-control kernel, until every stop flag of `lc` is set or `cap`
// iterations have run; the host launches it once and waits. The instantiated
// graph is cached in `cache` while its key and the contexts' buffers stay the same.
template <typename Capture>
acm_status graph_loop_run(GraphCache& cache, const GraphKey& key, std::vector<acm_ctx*>& ctxs, Capture&& capture,
                          LoopCtl lc, cudaStream_t st) {
  if (!(cache.exec && cache.key == key)) {
    if (cache.exec) {
      cudaGraphExecDestroy(cache.exec);
      cache.exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    CK(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle handle;
    const cudaError_t eh = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
    if (eh != cudaSuccess) {
      note_error(eh, "cudaGraphConditionalHandleCreate", __LINE__);
      cudaGraphDestroy(graph);
      cudaGetLastError();
      return ACM_ERR_CUDA;
    }
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = handle;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    const cudaError_t en = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
    if (en != cudaSuccess) {
      note_error(en, "cudaGraphAddNode(conditional while)", __LINE__);
      cudaGraphDestroy(graph);
      cudaGetLastError();
      return ACM_ERR_CUDA;
    }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    // capture on a private non-blocking stream (the caller's stream may be the
    // legacy default stream, which cannot be captured); every context launches
    // on it during the capture
    cudaStream_t capst = ctxs[0]->cap;
    if (!capst) {
      cudaGraphDestroy(graph);
      return ACM_ERR_CUDA;
    }
    std::vector<cudaStream_t> saved;
    for (acm_ctx* x : ctxs) {
      saved.push_back(x->st);
      x->st = capst;
    }
    const cudaError_t eb = cudaStreamBeginCaptureToGraph(capst, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (eb != cudaSuccess) {
      for (size_t i = 0; i < ctxs.size(); ++i) ctxs[i]->st = saved[i];
      note_error(eb, "cudaStreamBeginCaptureToGraph", __LINE__);
      cudaGraphDestroy(graph);
      cudaGetLastError();
      return ACM_ERR_CUDA;
    }
    acm_status s = capture();
    lc.counter = cache.counter;
    lc.cap = key.cap;
    lc.handle = handle;
    if (s == ACM_OK) {
      const cudaError_t el = loop_control(lc, capst);
      if (el != cudaSuccess) {
        note_error(el, "loop_control", __LINE__);
        s = ACM_ERR_CUDA;
      }
    }
    cudaGraph_t captured = body;
    const cudaError_t e = cudaStreamEndCapture(capst, &captured);
    for (size_t i = 0; i < ctxs.size(); ++i) ctxs[i]->st = saved[i];
    if (s != ACM_OK || e != cudaSuccess) {
      if (e != cudaSuccess) note_error(e, "cudaStreamEndCapture", __LINE__);
      cudaGraphDestroy(graph);
      cudaGetLastError();
      return s != ACM_OK ? s : ACM_ERR_CUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&cache.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      note_error(ei, "cudaGraphInstantiate", __LINE__);
      cudaGetLastError();
      cache.exec = nullptr;
      return ACM_ERR_CUDA;
    }
    cache.key = key;
  }
  CK(cudaMemsetAsync(cache.counter, 0, sizeof(unsigned int), st));
  CK(cudaGraphLaunch(cache.exec, st));
  CK(cudaStreamSynchronize(st));
  return ACM_OK;
}

// The Stokes loop of every group as one device-resident graph: [step 1, steps 2-4].
template <typename T>
acm_status stokes_graph_run(std::vector<StokesGroup>& grp, int deriv, unsigned cap, GraphCache& cache,
                            cudaStream_t st) {
  GraphKey key;
  key.prec = (int)sizeof(T);
  key.nprob = 0;
  for (auto& x : grp) key.nprob += x.nprob;
  key.deriv = deriv;
  key.kind = 1;
  key.cap = cap;
  std::vector<acm_ctx*> ctxs;
  LoopCtl lc = {};
  for (size_t i = 0; i < grp.size(); ++i) {
    ctxs.push_back(grp[i].c);
    lc.base[i] = (const char*)grp[i].c->sprm;
    lc.n[i] = grp[i].nprob;
    lc.stride[i] = (int)sizeof(StokesDev);
  }
  lc.ngroups = (int)grp.size();
  lc.done_off = (int)offsetof(StokesDev, done);
  auto capture = [&]() -> acm_status {
    acm_status s = ACM_OK;
    for (size_t i = 0; i < grp.size() && s == ACM_OK; ++i) {
      StokesGroup& x = grp[i];
      const Sym<T> sym = sym_of<T>(x.c, deriv);
      s = stokes_step1<T>(x.c, x.nprob, x.H, x.hs, x.lph, sym);
      if (s == ACM_OK) s = stokes_body<T>(x.c, x.nprob, x.H, x.hs, x.lph, sym, true);
    }
    return s;
  };
  return graph_loop_run(cache, key, ctxs, capture, lc, st);
}

// Iterations of the device-resident loop. With device_loop (and the profiler
// off) the whole loop is one graph launch; otherwise the host launches chunks
// of `check_every` iterations, reads the stop flags between chunks and never
// launches past `remaining`; problems that converge earlier turn the rest of
// their launches into immediate returns.
template <typename T>
acm_status stokes_iterate(acm_ctx* c, int nprob, const uint8_t* Hdev, long long hs, int lph, int deriv,
                          int check_every, int remaining, bool device_loop) {
  if (remaining <= 0) return ACM_OK;
  if (device_loop && !c->prof) {
    std::vector<StokesGroup> grp = {{c, nprob, Hdev, hs, lph}};
    return stokes_graph_run<T>(grp, deriv, (unsigned)remaining, c->graph, c->st);
  }
  const Sym<T> sym = sym_of<T>(c, deriv);
  CKS(stokes_step1<T>(c, nprob, Hdev, hs, lph, sym));
  CKS(pin_scratch(c, (size_t)c->B * sizeof(StokesDev)));
  if (check_every < 1) check_every = 1;
  while (remaining > 0) {
    const int chunk = check_every < remaining ? check_every : remaining;
    for (int k = 0; k < chunk; ++k) CKS(stokes_body<T>(c, nprob, Hdev, hs, lph, sym, remaining - k <= 1));
    remaining -= chunk;
    CK(cudaMemcpyAsync(c->pin, c->sprm, nprob * sizeof(StokesDev), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    const StokesDev* hp = (const StokesDev*)c->pin;
    bool all = true;
    for (int p = 0; p < nprob; ++p) all = all && hp[p].done;
    if (all) break;
  }
  return ACM_OK;
}

// continue an FP32 solve in FP64: convert the state, re-arm the stop flags
acm_status stokes_promote(acm_ctx* c, int nprob, double eps) {
  CKS(ensure_prec<double>(c));
  Prec& f = c->pf;
  Prec& d = c->pd;
  const Geo& g = c->g;
  LK(ACM_K_OTHER, convert_f2d((const float*)f.u, (double*)d.u, (long long)nprob * 3 * g.V, c->st));
  LK(ACM_K_OTHER, convert_f2d((const float*)f.lam, (double*)d.lam, (long long)nprob * 3 * g.V, c->st));
  LK(ACM_K_OTHER, convert_f2d((const float*)f.st0, (double*)d.st0, (long long)nprob * 2 * g.S, c->st));
  LK(ACM_K_OTHER, convert_f2d((const float*)f.st1, (double*)d.st1, (long long)nprob * 2 * g.S, c->st));
  std::vector<StokesDev> hp(nprob);
  CK(cudaMemcpyAsync(hp.data(), c->sprm, nprob * sizeof(StokesDev), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  for (auto& x : hp) {
    x.done = 0;
    x.converged = 0;
    x.status = 0;
    x.eps = eps;
    x.stall_win = 0;
  }
  CK(cudaMemcpyAsync(c->sprm, hp.data(), nprob * sizeof(StokesDev), cudaMemcpyHostToDevice, c->st));
  return ACM_OK;
}

template <typename T>
acm_status stokes_outputs(acm_ctx* c, int nprob, void* u_out, long long u_stride, void* p_out, void* lam_out,
                          double (*Kcol)[3]) {
  Prec& w = prec<T>(c);
  Geo g = c->g;
  g.us = 3 * g.V;
  g.hs = 0;
  for (int p = 0; p < nprob; ++p) {
    if (u_out)
      CK(cudaMemcpyAsync((char*)u_out + (size_t)p * u_stride * sizeof(T), (T*)w.u + (size_t)p * 3 * g.V,
                         3 * g.V * sizeof(T), cudaMemcpyDefault, c->st));
    if (lam_out)
      CK(cudaMemcpyAsync((char*)lam_out + (size_t)p * 3 * g.V * sizeof(T), (T*)w.lam + (size_t)p * 3 * g.V,
                         3 * g.V * sizeof(T), cudaMemcpyDefault, c->st));
  }
  if (p_out) {
    CKS(ensure_aux<T>(c));
    // p = q - mean(q): inverse transform of q^ (its k = 0 coefficient is 0)
    const Sym<T> sym = sym_of<T>(c, 0);
    LK(ACM_K_OTHER, Ops<T>::pass(g, 0, P_INV_SCALE, 1, nprob, w.st0, g.S, sym, w.tw, nullptr, nullptr, nullptr, nullptr, nullptr,
                    c->st));
    LK(ACM_K_OTHER, Ops<T>::pass(g, 1, P_INV, 1, nprob, w.st0, g.S, sym, w.tw, nullptr, nullptr, nullptr, nullptr, nullptr, c->st));
    LK(ACM_K_OTHER, Ops<T>::x_c2r(g, nprob, 1, w.st0, g.S, w.aux, g.V, w.tw, c->st));
    CK(cudaMemcpyAsync(p_out, w.aux, (size_t)nprob * g.V * sizeof(T), cudaMemcpyDefault, c->st));
  }
  if (Kcol) {
    g.hs = 0;
    LK(ACM_K_OTHER, Ops<T>::field_sums(g, nprob, w.u, c->Hd, c->part_r, NRED, c->st));
    std::vector<double> s;
    CKS(read_partials(c, nprob, 3, s));
    for (int p = 0; p < nprob; ++p)
      for (int k = 0; k < 3; ++k) Kcol[p][k] = s[(size_t)p * 3 + k] / (double)g.V;
  }
  CK(cudaStreamSynchronize(c->st));
  return ACM_OK;
}

// fp64_from: -1 all FP32, -2 all FP64, >= 0 mixed with it32[p] FP32 iterations of problem p
acm_status stokes_reports(acm_ctx* c, int nprob, acm_report* rep, int fp64_from, double t0,
                          const std::vector<int>* it32 = nullptr) {
  std::vector<StokesDev> hp(nprob);
  CK(cudaMemcpyAsync(hp.data(), c->sprm, nprob * sizeof(StokesDev), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  const double t1 = now_ms();
  acm_status worst = ACM_OK;
  for (int p = 0; p < nprob; ++p) {
    const StokesDev& d = hp[p];
    if (rep) {
      acm_report& r = rep[p];
      std::memset(&r, 0, sizeof(r));
      r.iters = d.iter;
      r.iters_fp64 = fp64_from >= 0 ? d.iter - (it32 ? (*it32)[p] : fp64_from) : (fp64_from == -2 ? d.iter : 0);
      r.converged = d.converged;
      r.status = d.status;
      for (int k = 0; k < 6; ++k) {
        r.res[k] = d.res[k];
        r.tol[k] = d.tol[k];
      }
      for (int k = 0; k < 3; ++k) r.psi[k] = d.psi_last[k];
      r.time_ms = t1 - t0;
    }
    if (d.status != ACM_OK && worst == ACM_OK) worst = (acm_status)d.status;
  }
  c->hist_kind = 1;
  for (int p = 0; p < nprob && p < BMAX; ++p) c->hist_n[p] = hp[p].iter < HIST_CAP ? hp[p].iter : HIST_CAP;
  return worst;
}

acm_status check_stokes_args(const acm_stokes_params& P) {
  if (!(P.nu > 0) || !(P.eps >= 0) || P.max_iter < 1 || (P.device_loop != 0 && P.device_loop != 1) || (P.deriv != 0 && P.deriv != 1) || P.precision < 0 ||
      P.precision > 2 || !(P.psi_min_frac > 0) || !(P.eps32 > 0) || !(P.pore_scale >= 0) ||
      !std::isfinite(P.pore_scale))
    return ACM_ERR_ARG;
  for (int k = 0; k < 3; ++k)
    if (!(P.phi[k] >= 1.0) || !(P.tau[k] >= 1.0)) return ACM_ERR_ARG;
  return ACM_OK;
}

// solve nprob loads on one H; u_out stride in elements between loads
acm_status stokes_solve(acm_ctx* c, int nprob, const uint8_t* H, const double (*gs)[3], const acm_stokes_params* prm,
                        const void* init_u, const void* init_lam, void* u_out, long long u_stride, void* p_out,
                        void* lam_out, double (*Kcol)[3], acm_report* rep) {
  acm_stokes_params P;
  fill_stokes_params(prm, &P);
  CKS(check_stokes_args(P));
  const double t0 = now_ms();
  const uint8_t* Hdev = nullptr;
  long long nsolid = 0;
  CKS(stage_H(c, H, &Hdev, &nsolid));
  if (nsolid == 0) return ACM_ERR_NO_SOLID;
  if (nsolid == c->g.V) return ACM_ERR_NO_FLUID;
  if (Hdev != c->Hd) CK(cudaMemcpyAsync(c->Hd, Hdev, (size_t)c->g.V, cudaMemcpyDeviceToDevice, c->st));
  Hdev = c->Hd;  // one stable buffer, so a cached device loop stays valid
  LK(ACM_K_OTHER, pack_hbits(c->Hd, c->Hb, c->g.V, c->st));
  std::vector<double> pore_l(nprob, 0.0);
  if (P.pore_scale > 0) {
    CK(cudaMemsetAsync(c->cnt, 0, sizeof(unsigned long long), c->st));
    LK(ACM_K_OTHER, count_faces_add(c->Hd, c->n0, c->n1, c->n2, c->cnt, c->st));
    CK(cudaMemcpyAsync(c->pin, c->cnt, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    const double faces = (double)*(unsigned long long*)c->pin;
    for (auto& x : pore_l) x = (double)(c->g.V - nsolid) / faces;
  }
  const bool dl = P.device_loop != 0;
  acm_status st = ACM_OK;
  const std::vector<const void*> iu(nprob, init_u), il(nprob, init_lam);
  if (P.precision == ACM_FP32) {
    CKS(stokes_setup<float>(c, nprob, Hdev, 0, 1, gs, P, P.eps, iu.data(), il.data(), nullptr, 0, pore_l.data()));
    CKS(stokes_iterate<float>(c, nprob, Hdev, 0, 1, P.deriv, P.check_every, P.max_iter, dl));
    CKS(stokes_outputs<float>(c, nprob, u_out, u_stride, p_out, lam_out, Kcol));
    st = stokes_reports(c, nprob, rep, -1, t0);
  } else if (P.precision == ACM_FP64) {
    CKS(stokes_setup<double>(c, nprob, Hdev, 0, 1, gs, P, P.eps, iu.data(), il.data(), nullptr, 0, pore_l.data()));
    CKS(stokes_iterate<double>(c, nprob, Hdev, 0, 1, P.deriv, P.check_every, P.max_iter, dl));
    CKS(stokes_outputs<double>(c, nprob, u_out, u_stride, p_out, lam_out, Kcol));
    st = stokes_reports(c, nprob, rep, -2, t0);
  } else {
    // FP32 iterations to eps32 (warm start given in double is cast on the host side by the caller)
    const double e32 = P.eps < P.eps32 ? P.eps32 : P.eps;
    if (init_u || init_lam) return ACM_ERR_ARG;  // warm starts are taken in the FP32 or FP64 modes
    CKS(stokes_setup<float>(c, nprob, Hdev, 0, 1, gs, P, e32, nullptr, nullptr, nullptr, STALL_WINDOW,
                            pore_l.data()));
    CKS(stokes_iterate<float>(c, nprob, Hdev, 0, 1, P.deriv, P.check_every, P.max_iter, dl));
    std::vector<StokesDev> hp(nprob);
    CK(cudaMemcpy(hp.data(), c->sprm, nprob * sizeof(StokesDev), cudaMemcpyDeviceToHost));
    // FP32 iterations of each problem; the host loop may run until the problem
    // with the fewest reaches the cap (the device stops each one at its own)
    std::vector<int> it32(nprob);
    int it32_min = P.max_iter;
    bool ok = true;
    for (int p = 0; p < nprob; ++p) {
      it32[p] = hp[p].iter;
      it32_min = std::min(it32_min, it32[p]);
      // a problem stopped at the FP32 rounding floor continues in FP64
      ok = ok && (hp[p].status == ACM_OK || hp[p].status == ST_STALLED);
    }
    if (ok && P.eps < e32) {
      CKS(stokes_promote(c, nprob, P.eps));
      CKS(stokes_iterate<double>(c, nprob, Hdev, 0, 1, P.deriv, P.check_every, P.max_iter - it32_min, dl));
      CKS(stokes_outputs<double>(c, nprob, u_out, u_stride, p_out, lam_out, Kcol));
      st = stokes_reports(c, nprob, rep, 0, t0, &it32);
    } else {
      // nothing left for FP64: report the FP32 result converted to the caller's double buffers
      CKS(stokes_promote(c, nprob, P.eps));
      CKS(stokes_outputs<double>(c, nprob, u_out, u_stride, p_out, lam_out, Kcol));
      std::vector<StokesDev> h2 = hp;
      CK(cudaMemcpy(c->sprm, h2.data(), nprob * sizeof(StokesDev), cudaMemcpyHostToDevice));
      st = stokes_reports(c, nprob, rep, -1, t0);
    }
  }
  return st;
}

// Eq. 2 literally: K_ij = h^3 sum over pore voxels of grad u^i : grad u^j, with the
// spectral gradient of the solve's derivative symbol; u^i in the Stokes state.
template <typename T>
acm_status perm_grad(acm_ctx* c, const uint8_t* Hdev, int deriv, double Kg[9]) {
  Prec& w = prec<T>(c);
  const Geo& g = c->g;
  const Sym<T> sym = sym_of<T>(c, deriv);
  const size_t cs = 2 * sizeof(T);
  CKS(ensure_aux<T>(c));
  T* f = (T*)w.aux;
  double K[6] = {0, 0, 0, 0, 0, 0};
  for (int l = 0; l < 3; ++l) {
    LK(ACM_K_OTHER, Ops<T>::x_r2c(g, 3, 1, w.st0, g.S, (T*)w.u + (size_t)l * g.V, 3 * g.V, w.tw, c->st));
    LK(ACM_K_OTHER, Ops<T>::pass(g, 1, P_FWD, 1, 3, w.st0, g.S, sym, w.tw, 0, 0, 0, 0, 0, c->st));
    for (int m = 0; m < 3; ++m) {
      CK(cudaMemcpyAsync(w.spec, w.st0, 3 * g.S * cs, cudaMemcpyDeviceToDevice, c->st));
      LK(ACM_K_OTHER, Ops<T>::pass(g, 0, P_DERIV, 1, 3, w.spec, g.S, sym, w.tw, 0, 0, 0, 0, 0, c->st, m));
      LK(ACM_K_OTHER, Ops<T>::pass(g, 1, P_INV, 1, 3, w.spec, g.S, sym, w.tw, 0, 0, 0, 0, 0, c->st));
      LK(ACM_K_OTHER, Ops<T>::x_c2r(g, 3, 1, w.spec, g.S, f, g.V, w.tw, c->st));
      LK(ACM_K_OTHER, Ops<T>::pore_products(g, f, Hdev, c->part_r, NRED, c->st));
      std::vector<double> s;
      CKS(read_partials(c, 1, 6, s));
      for (int k = 0; k < 6; ++k) K[k] += s[k];
    }
  }
  const int map[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Kg[i * 3 + j] = K[map[i][j]] / (double)g.V;
  return ACM_OK;
}

// ---------------------------------------------------------------------------
// solute (Section 3.2, Algorithm 1 Problem 2)
// ---------------------------------------------------------------------------
// One solute iteration of nprob problems (Algorithm 1, Problem 2): the x pass
// with the local terms of Eq. 18, the y forward pass, the z pass with Eq. 20
// and the Eq. 19 residuals, the y inverse pass, and the FP64 finalize.
template <typename T>
acm_status solute_body(acm_ctx* c, int nprob, const uint8_t* Hdev, const void* udev, long long us, const Sym<T>& sym) {
  Prec& w = prec<T>(c);
  Geo g = c->g;
  g.hs = 0;
  g.us = us;
  const int nbz = Ops<T>::z_blocks(g, P_SOLUTE);
  const long long ps = 4 * g.S;
  // spectral components per problem: x -> (tau_0, tau_1, s + d2 tau_2), y forward -> (tau_0, s''),
  // z -> (d0 chi, chi), y inverse -> (d0 chi, d1 chi, d2 chi)
  LK(ACM_K_X_SOLUTE, Ops<T>::x_solute(g, nprob, w.spec, udev, Hdev, c->Hb, c->cprm, w.tw, sym,
                                     c->solute_deriv == ACM_DERIV_CENTRAL, c->st));
  LK(ACM_K_Y_FWD_SOLUTE, Ops<T>::pass(g, 1, P_FWD_SOL, 3, nprob, w.spec, ps, sym, w.tw, nullptr, nullptr, nullptr, c->cprm,
                                     nullptr, c->st));
  LK(ACM_K_Z_SOLUTE, Ops<T>::pass(g, 0, P_SOLUTE, 2, nprob, w.spec, ps, sym, w.tw, w.st0, nullptr, nullptr, c->cprm,
                                  c->part_z, c->st));
  LK(ACM_K_Y_INV_SOLUTE, Ops<T>::pass(g, 1, P_INV_SOL, 3, nprob, w.spec, ps, sym, w.tw, nullptr, nullptr, nullptr, c->cprm,
                                     nullptr, c->st));
  LK(ACM_K_FINALIZE, solute_finalize(nprob, c->cprm, c->part_z, nbz, (double)g.V, c->hist, HIST_CAP, c->st));
  return ACM_OK;
}

// stall_win > 0: an FP32 phase that stops at its rounding floor (see StokesDev)
template <typename T>
acm_status solute_run(acm_ctx* c, int nprob, const uint8_t* Hdev, const void* udev, long long us,
                      const double (*gchi)[3], double Pe, const acm_advdiff_params& P, double eps, bool setup,
                      const double* B0, const double* ubar, int iters_done = 0, int stall_win = 0) {
  CKS(ensure_prec<T>(c));
  Prec& w = prec<T>(c);
  const Geo& g = c->g;
  const size_t cs = 2 * sizeof(T);
  const Sym<T> sym = sym_of<T>(c, P.deriv);
  c->solute_deriv = P.deriv;
  if (setup) {
    CK(cudaMemsetAsync(w.st0, 0, (size_t)nprob * g.S * cs, c->st));
    CK(cudaMemsetAsync(w.spec, 0, (size_t)nprob * 4 * g.S * cs, c->st));
    std::vector<SoluteDev> hp(nprob);
    for (int p = 0; p < nprob; ++p) {
      SoluteDev& d = hp[p];
      std::memset(&d, 0, sizeof(d));
      d.eps = eps;
      d.A0 = P.A0;
      d.eta = P.eta;
      d.Pe = Pe;
      double ug = 0;
      for (int k = 0; k < 3; ++k) {
        d.B0[k] = B0[k];
        d.g[k] = gchi[p][k];
        d.ubar[k] = ubar[k];
        ug += ubar[k] * gchi[p][k];
      }
      d.Fc = Pe * ug;
      d.max_iter = P.max_iter;
      d.rmin = 1e300;
      d.stall_win = stall_win;
      d.stall_best = 1e300;
    }
    CK(cudaMemcpyAsync(c->cprm, hp.data(), nprob * sizeof(SoluteDev), cudaMemcpyHostToDevice, c->st));
  }
  int remaining = P.max_iter - (setup ? 0 : iters_done);
  if (remaining <= 0) return ACM_OK;
  if (P.device_loop && !c->prof) {
    // the whole loop as one device-resident graph launch
    GraphKey key;
    key.prec = (int)sizeof(T);
    key.nprob = nprob;
    key.deriv = P.deriv;
    key.kind = 2;
    key.cap = (unsigned)remaining;
    key.kp = udev;
    key.kq = Hdev;
    key.kx = us;
    std::vector<acm_ctx*> ctxs = {c};
    LoopCtl lc = {};
    lc.base[0] = (const char*)c->cprm;
    lc.n[0] = nprob;
    lc.stride[0] = (int)sizeof(SoluteDev);
    lc.ngroups = 1;
    lc.done_off = (int)offsetof(SoluteDev, done);
    auto capture = [&]() -> acm_status { return solute_body<T>(c, nprob, Hdev, udev, us, sym); };
    return graph_loop_run(c->graph_sol, key, ctxs, capture, lc, c->st);
  }
  // host-launched chunks of check_every iterations; the stop flags are read between chunks
  CKS(pin_scratch(c, (size_t)c->B * sizeof(SoluteDev)));
  const int ce = P.check_every < 1 ? 1 : P.check_every;
  while (remaining > 0) {
    const int chunk = ce < remaining ? ce : remaining;
    remaining -= chunk;
    for (int k = 0; k < chunk; ++k) CKS(solute_body<T>(c, nprob, Hdev, udev, us, sym));
    CK(cudaMemcpyAsync(c->pin, c->cprm, nprob * sizeof(SoluteDev), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    const SoluteDev* hp = (const SoluteDev*)c->pin;
    bool all = true;
    for (int p = 0; p < nprob; ++p) all = all && hp[p].done;
    if (all) break;
  }
  return ACM_OK;
}

template <typename T>
acm_status solute_outputs(acm_ctx* c, int nprob, const uint8_t* Hdev, const void* udev, long long us, void* chi_out,
                          void* grad_out, double (*Dg)[3], double (*Dx)[3]) {
  Prec& w = prec<T>(c);
  Geo g = c->g;
  g.hs = 0;
  g.us = us;
  const Sym<T> sym = sym_of<T>(c, 0);
  CKS(ensure_aux<T>(c));
  T* grad = (T*)w.aux;
  T* chi = (T*)w.aux + (size_t)c->B * 3 * g.V;
  // grad chi^{n+1}: the last passes left i d0 chi^, i d1 chi^ and i d2 chi^ (inverse
  // along z and y) in components 0..2
  LK(ACM_K_OTHER, Ops<T>::x_c2r(g, nprob, 3, w.spec, 4 * g.S, grad, 3 * g.V, w.tw, c->st));
  // chi^{n+1}
  LK(ACM_K_OTHER, Ops<T>::pass(g, 0, P_INV_SCALE, 1, nprob, w.st0, g.S, sym, w.tw, nullptr, nullptr, nullptr, nullptr, nullptr,
                  c->st));
  LK(ACM_K_OTHER, Ops<T>::pass(g, 1, P_INV, 1, nprob, w.st0, g.S, sym, w.tw, nullptr, nullptr, nullptr, nullptr, nullptr, c->st));
  LK(ACM_K_OTHER, Ops<T>::x_c2r(g, nprob, 1, w.st0, g.S, chi, g.V, w.tw, c->st));
  LK(ACM_K_OTHER, Ops<T>::diffusivity(g, nprob, chi, grad, udev, Hdev, c->cprm, c->part_r, NRED, c->st));
  std::vector<double> s;
  CKS(read_partials(c, nprob, 6, s));
  for (int p = 0; p < nprob; ++p)
    for (int k = 0; k < 3; ++k) {
      Dg[p][k] = s[(size_t)p * 6 + k] / (double)g.V;
      if (Dx) Dx[p][k] = s[(size_t)p * 6 + 3 + k] / (double)g.V;
    }
  for (int p = 0; p < nprob; ++p) {
    if (chi_out)
      CK(cudaMemcpyAsync((T*)chi_out + (size_t)p * g.V, chi + (size_t)p * g.V, g.V * sizeof(T), cudaMemcpyDefault,
                         c->st));
    if (grad_out)
      CK(cudaMemcpyAsync((T*)grad_out + (size_t)p * 3 * g.V, grad + (size_t)p * 3 * g.V, 3 * g.V * sizeof(T),
                         cudaMemcpyDefault, c->st));
  }
  CK(cudaStreamSynchronize(c->st));
  return ACM_OK;
}

acm_status solute_promote(acm_ctx* c, int nprob, double eps) {
  CKS(ensure_prec<double>(c));
  const Geo& g = c->g;
  LK(ACM_K_OTHER, convert_f2d((const float*)c->pf.st0, (double*)c->pd.st0, (long long)nprob * 2 * g.S, c->st));
  LK(ACM_K_OTHER, convert_f2d((const float*)c->pf.spec, (double*)c->pd.spec, (long long)nprob * 4 * 2 * g.S, c->st));
  std::vector<SoluteDev> hp(nprob);
  CK(cudaMemcpyAsync(hp.data(), c->cprm, nprob * sizeof(SoluteDev), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  for (auto& x : hp) {
    x.done = 0;
    x.converged = 0;
    x.status = 0;
    x.eps = eps;
    x.stall_win = 0;
  }
  CK(cudaMemcpyAsync(c->cprm, hp.data(), nprob * sizeof(SoluteDev), cudaMemcpyHostToDevice, c->st));
  return ACM_OK;
}

// it32: FP32 iterations of each problem of a mixed solve (nullptr: no FP64 stage)
acm_status solute_reports(acm_ctx* c, int nprob, acm_report* rep, const std::vector<int>* it32, bool fp64_all,
                          double t0) {
  std::vector<SoluteDev> hp(nprob);
  CK(cudaMemcpyAsync(hp.data(), c->cprm, nprob * sizeof(SoluteDev), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  const double t1 = now_ms();
  acm_status worst = ACM_OK;
  for (int p = 0; p < nprob; ++p) {
    const SoluteDev& d = hp[p];
    if (rep) {
      acm_report& r = rep[p];
      std::memset(&r, 0, sizeof(r));
      r.iters = d.iter;
      r.iters_fp64 = fp64_all ? d.iter : (it32 ? d.iter - (*it32)[p] : 0);
      r.converged = d.converged;
      r.status = d.status;
      r.res[0] = d.res[0];
      r.res[1] = d.res[1];
      r.tol[0] = d.tol[0];
      r.tol[1] = d.tol[1];
      r.time_ms = t1 - t0;
    }
    if (d.status != ACM_OK && worst == ACM_OK) worst = (acm_status)d.status;
  }
  c->hist_kind = 2;
  for (int p = 0; p < nprob && p < BMAX; ++p) c->hist_n[p] = hp[p].iter < HIST_CAP ? hp[p].iter : HIST_CAP;
  return worst;
}

acm_status advdiff_solve(acm_ctx* c, int nprob, const uint8_t* H, const void* u, double Pe, const double (*gchi)[3],
                         const acm_advdiff_params* prm, void* chi_out, void* grad_out, double (*Dg)[3],
                         double (*Dx)[3], acm_report* rep) {
  acm_advdiff_params P;
  acm_advdiff_default_params(&P);
  if (prm) P = *prm;
  if (!u || !(P.A0 > 0) || !(P.eta >= 0) || !(P.eps >= 0) || P.max_iter < 1 || (P.deriv != 0 && P.deriv != 1) ||
      P.precision < 0 || P.precision > 2 || !std::isfinite(Pe) || (P.device_loop != 0 && P.device_loop != 1))
    return ACM_ERR_ARG;
  const double t0 = now_ms();
  const uint8_t* Hdev = nullptr;
  long long nsolid = 0;
  CKS(stage_H(c, H, &Hdev, &nsolid));
  LK(ACM_K_OTHER, pack_hbits(Hdev, c->Hb, c->g.V, c->st));
  if (nsolid == c->g.V) return ACM_ERR_NO_FLUID;
  const bool fp32 = P.precision == ACM_FP32;
  const size_t rs = fp32 ? sizeof(float) : sizeof(double);
  const Geo& g0 = c->g;
  // the advecting velocity in device memory of the working precision, used in
  // place when it is a 16-byte aligned device buffer (the x pass reads voxel
  // pairs as vectors and prefetches whole rows into L2 in 16-byte units)
  const void* ud = u;
  const bool in_place = is_device_ptr(u) && ((uintptr_t)u % 16) == 0;
  if (fp32) {
    CKS(ensure_prec<float>(c));
    if (!in_place) {
      CK(cudaMemcpyAsync(c->pf.u, u, 3 * g0.V * rs, cudaMemcpyDefault, c->st));
      ud = c->pf.u;
    }
  } else {
    CKS(ensure_prec<double>(c));
    if (!in_place) {
      CK(cudaMemcpyAsync(c->pd.u, u, 3 * g0.V * rs, cudaMemcpyDefault, c->st));
      ud = c->pd.u;
    }
  }
  // pore average of u (definition below Eq. 1) and the default comparison medium B0
  Geo g = g0;
  g.us = 0;
  g.hs = 0;
  std::vector<double> s;
  if (fp32) LK(ACM_K_OTHER, Ops<float>::field_sums(g, 1, ud, Hdev, c->part_r, NRED, c->st));
  else LK(ACM_K_OTHER, Ops<double>::field_sums(g, 1, ud, Hdev, c->part_r, NRED, c->st));
  {
    CKS(pin_scratch(c, (size_t)NRED * 8 * sizeof(double)));
    CK(cudaMemcpyAsync(c->pin, c->part_r, (size_t)NRED * 8 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    const double* h = (const double*)c->pin;
    s.assign(7, 0.0);
    for (int i = 0; i < NRED; ++i)
      for (int k = 0; k < 7; ++k) s[k] += h[(size_t)i * 8 + k];
  }
  const double npore = s[6];
  double ubar[3], B0[3];
  for (int k = 0; k < 3; ++k) {
    ubar[k] = s[3 + k] / npore;
    B0[k] = P.B0_explicit ? P.B0[k] : Pe * s[3 + k] / (double)g.V;
  }
  acm_status st = ACM_OK;
  if (P.precision == ACM_FP32) {
    CKS(solute_run<float>(c, nprob, Hdev, ud, 0, gchi, Pe, P, P.eps, true, B0, ubar));
    CKS(solute_outputs<float>(c, nprob, Hdev, ud, 0, chi_out, grad_out, Dg, Dx));
    st = solute_reports(c, nprob, rep, nullptr, false, t0);
  } else if (P.precision == ACM_FP64) {
    CKS(solute_run<double>(c, nprob, Hdev, ud, 0, gchi, Pe, P, P.eps, true, B0, ubar));
    CKS(solute_outputs<double>(c, nprob, Hdev, ud, 0, chi_out, grad_out, Dg, Dx));
    st = solute_reports(c, nprob, rep, nullptr, true, t0);
  } else {
    // FP32 phase needs the velocity in FP32
    CKS(ensure_prec<float>(c));
    LK(ACM_K_OTHER, convert_d2f((const double*)ud, (float*)c->pf.u, 3 * g.V, c->st));
    const double e32 = P.eps < 1e-5 ? 1e-5 : P.eps;
    CKS(solute_run<float>(c, nprob, Hdev, c->pf.u, 0, gchi, Pe, P, e32, true, B0, ubar, 0, STALL_WINDOW));
    std::vector<SoluteDev> hp(nprob);
    CK(cudaMemcpy(hp.data(), c->cprm, nprob * sizeof(SoluteDev), cudaMemcpyDeviceToHost));
    std::vector<int> it32(nprob);
    int it32_min = P.max_iter;
    bool ok = true;
    for (int p = 0; p < nprob; ++p) {
      it32[p] = hp[p].iter;
      it32_min = std::min(it32_min, it32[p]);
      // a problem stopped at the FP32 rounding floor continues in FP64
      ok = ok && (hp[p].status == ACM_OK || hp[p].status == ST_STALLED);
    }
    CKS(solute_promote(c, nprob, P.eps));
    const bool refine = ok && P.eps < e32;
    if (refine) CKS(solute_run<double>(c, nprob, Hdev, ud, 0, gchi, Pe, P, P.eps, false, B0, ubar, it32_min));
    else CK(cudaMemcpy(c->cprm, hp.data(), nprob * sizeof(SoluteDev), cudaMemcpyHostToDevice));
    CKS(solute_outputs<double>(c, nprob, Hdev, ud, 0, chi_out, grad_out, Dg, Dx));
    st = solute_reports(c, nprob, rep, refine ? &it32 : nullptr, false, t0);
  }
  return st;
}


// ---------------------------------------------------------------------------
// batched Stokes: many cells, three loads each; cells of one shape share every
// launch (one context per shape with room for 3 x cells problems)
// ---------------------------------------------------------------------------
struct BatchGroup {
  int n[3];
  std::vector<int> cells;
  acm_ctx* c = nullptr;
  std::vector<int> iters;  // iterations of each problem in the last solve
};

}  // namespace

struct acm_batch {
  cudaStream_t st = nullptr;
  int ncells = 0;
  std::vector<BatchGroup> groups;
  GraphCache graph;
  unsigned long long* counts = nullptr;  // device [2][ncells]: solid voxels, solid-pore faces
};

namespace {

template <typename T>
acm_status batch_stokes_run(acm_batch* b, const uint8_t* const* H, const acm_stokes_params& P,
                            const void* const* init_u, const void* const* init_lam, void* const* u_out,
                            void* const* lam_out, double* K, acm_report* rep) {
  const double t0 = now_ms();
  // indicators into each group's cell slots, solid counts per cell
  // counts[cell] = solid voxels, counts[ncells + cell] = solid-pore faces
  CK(cudaMemsetAsync(b->counts, 0, (size_t)2 * b->ncells * sizeof(unsigned long long), b->st));
  for (auto& gr : b->groups) {
    const long long V = gr.c->g.V;
    for (size_t i = 0; i < gr.cells.size(); ++i) {
      const int cell = gr.cells[i];
      if (!H[cell]) return ACM_ERR_ARG;
      CK(cudaMemcpyAsync(gr.c->Hd + i * V, H[cell], (size_t)V, cudaMemcpyDefault, b->st));
      CK(count_solid_add(gr.c->Hd + i * V, V, b->counts + cell, b->st));
      if (P.pore_scale > 0)
        CK(count_faces_add(gr.c->Hd + i * V, gr.n[0], gr.n[1], gr.n[2], b->counts + b->ncells + cell, b->st));
    }
    CK(pack_hbits(gr.c->Hd, gr.c->Hb, (long long)gr.cells.size() * V, b->st));
  }
  std::vector<unsigned long long> cnt(2 * (size_t)b->ncells);
  CK(cudaMemcpyAsync(cnt.data(), b->counts, cnt.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, b->st));
  CK(cudaStreamSynchronize(b->st));
  // per-problem set-up (degenerate cells are reported, not iterated)
  std::vector<StokesGroup> grp;
  for (auto& gr : b->groups) {
    const int nc = (int)gr.cells.size(), np = 3 * nc;
    const long long V = gr.c->g.V;
    std::vector<int> preset(np, ACM_OK);
    std::vector<double> gs((size_t)np * 3, 0.0);
    for (int p = 0; p < np; ++p) {
      const unsigned long long ns = cnt[gr.cells[p / 3]];
      preset[p] = ns == 0 ? ACM_ERR_NO_SOLID : (ns == (unsigned long long)V ? ACM_ERR_NO_FLUID : ACM_OK);
      gs[(size_t)p * 3 + p % 3] = 1.0;
    }
    // warm starts of the three loads of a cell lie 3 V apart in its buffer
    std::vector<const void*> iu(np, nullptr), il(np, nullptr);
    for (int p = 0; p < np; ++p) {
      const int cell = gr.cells[p / 3];
      const size_t off = (size_t)(p % 3) * 3 * V * sizeof(T);
      if (init_u && init_u[cell]) iu[p] = (const char*)init_u[cell] + off;
      if (init_lam && init_lam[cell]) il[p] = (const char*)init_lam[cell] + off;
    }
    std::vector<double> pore_l(np, 0.0);
    for (int p = 0; p < np; ++p) {
      const int cell = gr.cells[p / 3];
      const unsigned long long faces = cnt[(size_t)b->ncells + cell];
      if (faces > 0) pore_l[p] = (double)(V - (long long)cnt[cell]) / (double)faces;
    }
    CKS(stokes_setup<T>(gr.c, np, gr.c->Hd, V, 3, reinterpret_cast<const double(*)[3]>(gs.data()), P, P.eps,
                        iu.data(), il.data(), preset.data(), 0, pore_l.data()));
    grp.push_back({gr.c, np, gr.c->Hd, V, 3});
  }
  bool prof = false;
  for (auto& gr : b->groups) prof = prof || gr.c->prof;
  if (P.device_loop && !prof) {
    CKS(stokes_graph_run<T>(grp, P.deriv, (unsigned)P.max_iter, b->graph, b->st));
  } else {
    for (auto& x : grp)
      CKS(stokes_iterate<T>(x.c, x.nprob, x.H, x.hs, x.lph, P.deriv, P.check_every, P.max_iter, false));
  }
  // outputs: K per cell (volume averages of the three loads), fields, reports
  const double t1 = now_ms();
  for (auto& gr : b->groups) {
    acm_ctx* c = gr.c;
    Prec& w = prec<T>(c);
    Geo g = c->g;
    g.us = 3 * g.V;
    g.hs = 0;
    const int nc = (int)gr.cells.size(), np = 3 * nc;
    LK(ACM_K_OTHER, Ops<T>::field_sums(g, np, w.u, c->Hd, c->part_r, NRED, c->st));
    std::vector<double> sums;
    CKS(read_partials(c, np, 3, sums));
    std::vector<StokesDev> hp(np);
    CK(cudaMemcpyAsync(hp.data(), c->sprm, np * sizeof(StokesDev), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    gr.iters.assign(np, 0);
    for (int p = 0; p < np; ++p) gr.iters[p] = hp[p].iter;
    for (int i = 0; i < nc; ++i) {
      const int cell = gr.cells[i];
      for (int j = 0; j < 3; ++j) {
        const int p = 3 * i + j;
        for (int r = 0; r < 3; ++r)
          K[(size_t)cell * 9 + r * 3 + j] =
              hp[p].status == ACM_ERR_NO_SOLID || hp[p].status == ACM_ERR_NO_FLUID ? NAN : sums[(size_t)p * 3 + r] / (double)g.V;
        if (rep) {
          acm_report& R = rep[(size_t)cell * 3 + j];
          std::memset(&R, 0, sizeof(R));
          R.iters = hp[p].iter;
          R.iters_fp64 = sizeof(T) == 8 ? hp[p].iter : 0;
          R.converged = hp[p].converged;
          R.status = hp[p].status;
          for (int k = 0; k < 6; ++k) {
            R.res[k] = hp[p].res[k];
            R.tol[k] = hp[p].tol[k];
          }
          for (int k = 0; k < 3; ++k) R.psi[k] = hp[p].psi_last[k];
          R.time_ms = t1 - t0;
        }
      }
      if (u_out && u_out[cell])
        CK(cudaMemcpyAsync(u_out[cell], (T*)w.u + (size_t)3 * i * 3 * g.V, (size_t)9 * g.V * sizeof(T),
                           cudaMemcpyDefault, c->st));
      if (lam_out && lam_out[cell])
        CK(cudaMemcpyAsync(lam_out[cell], (T*)w.lam + (size_t)3 * i * 3 * g.V, (size_t)9 * g.V * sizeof(T),
                           cudaMemcpyDefault, c->st));
    }
  }
  CK(cudaStreamSynchronize(b->st));
  return ACM_OK;
}

// ---------------------------------------------------------------------------
// Tile autotuner: times each candidate tile width of the strided passes of the
// solver loops on this context's workspace (nprob problems, CUDA events on the
// context's stream) and keeps the fastest. The tile width only regroups which
// columns a block transforms, so every choice gives the same fields; only the
// order of the FP64 partial sums of the z pass changes.
// ---------------------------------------------------------------------------
struct TuneJob {
  int axis, op, nc;
  bool solute;
};
constexpr TuneJob TUNE_JOBS[] = {{1, P_FWD, 3, false},    {0, P_STOKES, 3, false}, {1, P_INV, 3, false},
                                 {1, P_FWD_SOL, 3, true}, {0, P_SOLUTE, 2, true},  {1, P_INV_SOL, 3, true}};
constexpr int NTUNE = (int)(sizeof(TUNE_JOBS) / sizeof(TUNE_JOBS[0]));
constexpr int TUNE_REPS = 5;

template <typename T>
acm_status autotune_ctx(acm_ctx* c, int nprob, int deriv) {
  CKS(ensure_prec<T>(c));
  Prec& w = prec<T>(c);
  const int pr = sizeof(T) == 8;
  // parameters that keep every pass from taking its early exit
  std::vector<StokesDev> sd(nprob);
  std::vector<SoluteDev> cd(nprob);
  for (int p = 0; p < nprob; ++p) {
    std::memset(&sd[p], 0, sizeof(StokesDev));
    std::memset(&cd[p], 0, sizeof(SoluteDev));
    sd[p].nu = 1.0;
    for (int k = 0; k < 3; ++k) {
      sd[p].psi[k] = 1.0;
      cd[p].B0[k] = 1.0;
    }
    cd[p].A0 = 0.55;
  }
  CK(cudaMemcpyAsync(c->sprm, sd.data(), nprob * sizeof(StokesDev), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->cprm, cd.data(), nprob * sizeof(SoluteDev), cudaMemcpyHostToDevice, c->st));
  const Sym<T> sym = sym_of<T>(c, deriv);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  acm_status st = ACM_OK;
  for (const TuneJob& j : TUNE_JOBS) {
    if (j.solute && c->spec_comps < 4) continue;
    const int n = j.axis == 1 ? c->g.n1 : c->g.n0;
    float best = 0;
    int best_sh = 0;
    for (int sh = -1; sh <= 4 && st == ACM_OK; ++sh) {   // 3, 4: the register-resident variants
      if (!Ops<T>::tx_variant(n, j.op, j.nc, sh)) continue;
      Geo g = c->g;
      g.txs[pr][j.axis][j.op] = (signed char)sh;
      const long long ps = (long long)j.nc * g.S;
      StokesDev* sp = j.solute ? nullptr : c->sprm;
      SoluteDev* cp = j.solute ? c->cprm : nullptr;
      void* s0 = j.op == P_STOKES || j.op == P_SOLUTE ? w.st0 : nullptr;
      void* s1 = j.op == P_STOKES ? w.st1 : nullptr;
      double* part = j.op == P_STOKES || j.op == P_SOLUTE ? c->part_z : nullptr;
      float ms = 0;
      for (int r = 0; r < 2 + TUNE_REPS && st == ACM_OK; ++r) {
        if (r == 2 && cudaEventRecord(e0, c->st) != cudaSuccess) st = ACM_ERR_CUDA;
        if (Ops<T>::pass(g, j.axis, j.op, j.nc, nprob, w.spec, ps, sym, w.tw, s0, s1, sp, cp, part, c->st) !=
            cudaSuccess)
          st = ACM_ERR_CUDA;
      }
      if (st == ACM_OK && (cudaEventRecord(e1, c->st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                           cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        st = ACM_ERR_CUDA;
      if (st == ACM_OK && (sh == -1 || best == 0 || ms < best)) {
        if (best == 0 || ms < best) {
          best = ms;
          best_sh = sh;
        }
      }
    }
    if (st != ACM_OK) break;
    c->g.txs[pr][j.axis][j.op] = (signed char)best_sh;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != ACM_OK) {
    cudaGetLastError();
    return st;
  }
  // a captured loop holds the old launches
  drop_graphs(c);
  CK(cudaStreamSynchronize(c->st));
  return ACM_OK;
}

// tile widths of the tuned passes (0 where a pass does not apply)
void tiles_of(const acm_ctx* c, int fp64, int tiles[NTUNE]) {
  for (int i = 0; i < NTUNE; ++i) {
    const TuneJob& j = TUNE_JOBS[i];
    tiles[i] = j.solute && c->spec_comps < 4
                   ? 0
                   : (fp64 ? Ops<double>::pass_tx(c->g, j.axis, j.op, j.nc) : Ops<float>::pass_tx(c->g, j.axis, j.op, j.nc));
  }
}

// A context for grids of one shape with room for B problems (loads) and
// `ncells` indicator grids (cells of a batch; problem p uses cell p / lph).
acm_status ctx_create(acm_ctx** out, int n0, int n1, int n2, void* stream, int B, int ncells) {
  if (!out || B < 1 || ncells < 1) return ACM_ERR_ARG;
  *out = nullptr;
  if (!shape_ok(n0, n1, n2)) return ACM_ERR_UNSUPPORTED_SIZE;
  acm_ctx* c = new (std::nothrow) acm_ctx();
  if (!c) return ACM_ERR_NOMEM;
  c->n0 = n0;
  c->n1 = n1;
  c->n2 = n2;
  c->B = B;
  c->ncells = ncells;
  Geo& g = c->g;
  g.n0 = n0;
  g.n1 = n1;
  g.n2 = n2;
  g.Pu = n2 / 2 + 1;
  g.P = n2 / 2 + 4;  // rows start on 32-byte sectors for both precisions
  g.V = (long long)n0 * n1 * n2;
  g.S = (long long)n0 * n1 * g.P;
  g.hs = 0;
  g.us = 3 * g.V;
  g.lph = 1;
  c->st = (cudaStream_t)stream;
  const int nbx = Ops<float>::x_blocks(g);
  // partial sums sized for the narrowest tile variant the autotuner may pick
  Geo gn = g;
  for (int pr = 0; pr < 2; ++pr)
    for (int ax = 0; ax < 2; ++ax)
      for (int op = 0; op < 8; ++op) gn.txs[pr][ax][op] = -1;
  const int nbz = std::max(std::max(Ops<float>::z_blocks(gn, P_STOKES), Ops<float>::z_blocks(gn, P_SOLUTE)),
                           std::max(Ops<double>::z_blocks(gn, P_STOKES), Ops<double>::z_blocks(gn, P_SOLUTE)));
  c->nbx = nbx;
  c->nbz = nbz;
  bool ok = cudaMalloc(&c->sprm, (size_t)B * sizeof(StokesDev)) == cudaSuccess &&
            cudaMalloc(&c->cprm, (size_t)B * sizeof(SoluteDev)) == cudaSuccess &&
            cudaMalloc(&c->part_x, (size_t)B * nbx * 8 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->part_z, (size_t)B * nbz * 4 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->part_r, (size_t)B * NRED * 8 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->Hd, (size_t)ncells * g.V) == cudaSuccess &&
            cudaMalloc(&c->Hb, (size_t)ncells * g.V / 8) == cudaSuccess &&
            cudaMalloc(&c->cnt, sizeof(unsigned long long)) == cudaSuccess &&
            cudaMalloc(&c->graph.counter, sizeof(unsigned int)) == cudaSuccess &&
            cudaMalloc(&c->graph_sol.counter, sizeof(unsigned int)) == cudaSuccess &&
            cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMalloc(&c->hist, (size_t)BMAX * HIST_CAP * STOKES_HIST * sizeof(double)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    acm_destroy(c);
    return ACM_ERR_NOMEM;
  }
  if (cudaMemset(c->sprm, 0, (size_t)B * sizeof(StokesDev)) != cudaSuccess ||
      cudaMemset(c->cprm, 0, (size_t)B * sizeof(SoluteDev)) != cudaSuccess) {
    cudaGetLastError();
    acm_destroy(c);
    return ACM_ERR_CUDA;
  }
  *out = c;
  return ACM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

acm_status acm_stokes_default_params(acm_stokes_params* p) {
  if (!p) return ACM_ERR_ARG;
  std::memset(p, 0, sizeof(*p));
  p->nu = 1.0;
  p->eps = 1e-5;
  p->alpha0 = p->beta0 = p->b0 = 0.0;
  for (int k = 0; k < 3; ++k) p->phi[k] = 1.1;
  p->tau[0] = 5.0;
  p->tau[1] = 10.0;
  p->tau[2] = 5.0;
  p->psi_min_frac = 1e-3;
  p->eps32 = 1e-5;
  p->max_iter = 20000;
  p->adaptive = 1;
  p->deriv = ACM_DERIV_EXACT;
  p->precision = ACM_FP32;
  p->check_every = 16;
  p->device_loop = 1;
  return ACM_OK;
}

acm_status acm_advdiff_default_params(acm_advdiff_params* p) {
  if (!p) return ACM_ERR_ARG;
  std::memset(p, 0, sizeof(*p));
  p->eta = 0.01;
  p->A0 = 0.55;
  p->B0_explicit = 0;
  p->eps = 1e-5;
  p->max_iter = 20000;
  p->deriv = ACM_DERIV_CENTRAL;
  p->precision = ACM_FP32;
  p->check_every = 16;
  p->device_loop = 1;
  return ACM_OK;
}

acm_status acm_create(acm_ctx** out, int n0, int n1, int n2, void* stream) {
  return ctx_create(out, n0, n1, n2, stream, BMAX, 1);
}

acm_status acm_destroy(acm_ctx* c) {
  if (!c) return ACM_ERR_ARG;
  if (c->st) cudaStreamSynchronize(c->st);
  else cudaDeviceSynchronize();
  free_prec(c->pf);
  free_prec(c->pd);
  drop_graphs(c);
  if (c->cap) cudaStreamDestroy(c->cap);
  void* ps[] = {c->sprm, c->cprm, c->part_x, c->part_z, c->part_r, c->Hd, c->Hb, c->cnt, c->hist, c->hist_b,
                c->graph.counter, c->graph_sol.counter};
  for (void* p : ps)
    if (p) cudaFree(p);
  if (c->pin) cudaFreeHost(c->pin);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  cudaGetLastError();
  delete c;
  return ACM_OK;
}

acm_status acm_stokes(acm_ctx* c, const uint8_t* H, const double g[3], const acm_stokes_params* prm,
                      const void* init_u, const void* init_lambda, void* u, void* p, void* lambda, double K_col[3],
                      acm_report* rep) {
  if (!c || !H || !g || !u) return ACM_ERR_ARG;
  double gs[1][3] = {{g[0], g[1], g[2]}};
  double K[1][3];
  acm_status s = stokes_solve(c, 1, H, gs, prm, init_u, init_lambda, u, 3 * c->g.V, p, lambda, K_col ? K : nullptr,
                              rep);
  if ((s == ACM_OK || s == ACM_ERR_MAXITER) && K_col)
    for (int k = 0; k < 3; ++k) K_col[k] = K[0][k];
  return s;
}

acm_status acm_stokes_tensor(acm_ctx* c, const uint8_t* H, const acm_stokes_params* prm, void* u3, double K[9],
                             double K_grad[9], acm_report rep[3]) {
  if (!c || !H || !K) return ACM_ERR_ARG;
  double gs[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  double Kc[3][3];
  acm_status s = stokes_solve(c, 3, H, gs, prm, nullptr, nullptr, u3, 3 * c->g.V, nullptr, nullptr, Kc, rep);
  if (s == ACM_OK || s == ACM_ERR_MAXITER) {
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) K[i * 3 + j] = Kc[j][i];
    if (K_grad) {
      acm_stokes_params P;
      fill_stokes_params(prm, &P);
      acm_status s2 = P.precision == ACM_FP32 ? perm_grad<float>(c, c->Hd, P.deriv, K_grad)
                                              : perm_grad<double>(c, c->Hd, P.deriv, K_grad);
      if (s2 != ACM_OK) return s2;
    }
  }
  return s;
}

acm_status acm_advdiff(acm_ctx* c, const uint8_t* H, const void* u, double Pe, const double g_chi[3],
                       const acm_advdiff_params* prm, void* chi, void* grad_chi, double Dg[3], double Dg_ext[3],
                       acm_report* rep) {
  if (!c || !H || !u || !g_chi || !Dg) return ACM_ERR_ARG;
  double gs[1][3] = {{g_chi[0], g_chi[1], g_chi[2]}};
  double D[1][3], Dx[1][3];
  acm_status s = advdiff_solve(c, 1, H, u, Pe, gs, prm, chi, grad_chi, D, Dx, rep);
  if (s == ACM_OK || s == ACM_ERR_MAXITER)
    for (int k = 0; k < 3; ++k) {
      Dg[k] = D[0][k];
      if (Dg_ext) Dg_ext[k] = Dx[0][k];
    }
  return s;
}

acm_status acm_advdiff_tensor(acm_ctx* c, const uint8_t* H, const void* u, double Pe, const acm_advdiff_params* prm,
                              void* chi3, double D[9], double D_ext[9], acm_report rep[3]) {
  if (!c || !H || !u || !D) return ACM_ERR_ARG;
  double gs[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  double Dc[3][3], Dx[3][3];
  acm_status s = advdiff_solve(c, 3, H, u, Pe, gs, prm, chi3, nullptr, Dc, Dx, rep);
  if (s == ACM_OK || s == ACM_ERR_MAXITER)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        D[i * 3 + j] = Dc[j][i];
        if (D_ext) D_ext[i * 3 + j] = Dx[j][i];
      }
  return s;
}

static acm_status fft_impl(acm_ctx* c, int fp64, int nbatch, const void* in, void* out, bool forward) {
  if (!c || !in || !out || nbatch < 1 || (fp64 != 0 && fp64 != 1)) return ACM_ERR_ARG;
  const Geo& g = c->g;
  const size_t rs = fp64 ? sizeof(double) : sizeof(float);
  const size_t cs = 2 * rs;
  if (fp64) CKS(ensure_aux<double>(c));
  else CKS(ensure_aux<float>(c));
  Prec& w = fp64 ? c->pd : c->pf;
  for (int b = 0; b < nbatch; ++b) {
    if (forward) {
      const void* src = (const char*)in + (size_t)b * g.V * rs;
      if (!is_device_ptr(in)) {
        CK(cudaMemcpyAsync(w.aux, src, g.V * rs, cudaMemcpyHostToDevice, c->st));
        src = w.aux;
      }
      if (fp64) {
        const Sym<double> sym = sym_of<double>(c, 0);
        LK(ACM_K_OTHER, Ops<double>::x_r2c(g, 1, 1, w.st0, g.S, src, g.V, w.tw, c->st));
        LK(ACM_K_OTHER, Ops<double>::pass(g, 1, P_FWD, 1, 1, w.st0, g.S, sym, w.tw, 0, 0, 0, 0, 0, c->st));
        LK(ACM_K_OTHER, Ops<double>::pass(g, 0, P_FWD, 1, 1, w.st0, g.S, sym, w.tw, 0, 0, 0, 0, 0, c->st));
      } else {
        const Sym<float> sym = sym_of<float>(c, 0);
        LK(ACM_K_OTHER, Ops<float>::x_r2c(g, 1, 1, w.st0, g.S, src, g.V, w.tw, c->st));
        LK(ACM_K_OTHER, Ops<float>::pass(g, 1, P_FWD, 1, 1, w.st0, g.S, sym, w.tw, 0, 0, 0, 0, 0, c->st));
        LK(ACM_K_OTHER, Ops<float>::pass(g, 0, P_FWD, 1, 1, w.st0, g.S, sym, w.tw, 0, 0, 0, 0, 0, c->st));
      }
      CK(cudaMemcpy2DAsync((char*)out + (size_t)b * g.n0 * g.n1 * g.Pu * cs, g.Pu * cs, w.st0, g.P * cs, g.Pu * cs,
                           (size_t)g.n0 * g.n1, cudaMemcpyDefault, c->st));
    } else {
      CK(cudaMemcpy2DAsync(w.st0, g.P * cs, (const char*)in + (size_t)b * g.n0 * g.n1 * g.Pu * cs, g.Pu * cs,
                           g.Pu * cs, (size_t)g.n0 * g.n1, cudaMemcpyDefault, c->st));
      void* dst = (char*)out + (size_t)b * g.V * rs;
      const bool dev = is_device_ptr(out);
      void* tgt = dev ? dst : w.aux;
      if (fp64) {
        const Sym<double> sym = sym_of<double>(c, 0);
        LK(ACM_K_OTHER, Ops<double>::pass(g, 0, P_INV_SCALE, 1, 1, w.st0, g.S, sym, w.tw, 0, 0, 0, 0, 0, c->st));
        LK(ACM_K_OTHER, Ops<double>::pass(g, 1, P_INV, 1, 1, w.st0, g.S, sym, w.tw, 0, 0, 0, 0, 0, c->st));
        LK(ACM_K_OTHER, Ops<double>::x_c2r(g, 1, 1, w.st0, g.S, tgt, g.V, w.tw, c->st));
      } else {
        const Sym<float> sym = sym_of<float>(c, 0);
        LK(ACM_K_OTHER, Ops<float>::pass(g, 0, P_INV_SCALE, 1, 1, w.st0, g.S, sym, w.tw, 0, 0, 0, 0, 0, c->st));
        LK(ACM_K_OTHER, Ops<float>::pass(g, 1, P_INV, 1, 1, w.st0, g.S, sym, w.tw, 0, 0, 0, 0, 0, c->st));
        LK(ACM_K_OTHER, Ops<float>::x_c2r(g, 1, 1, w.st0, g.S, tgt, g.V, w.tw, c->st));
      }
      if (!dev) CK(cudaMemcpyAsync(dst, w.aux, g.V * rs, cudaMemcpyDeviceToHost, c->st));
    }
  }
  CK(cudaStreamSynchronize(c->st));
  return ACM_OK;
}

acm_status acm_fft_r2c(acm_ctx* c, int fp64, int nbatch, const void* in, void* out) {
  return fft_impl(c, fp64, nbatch, in, out, true);
}

acm_status acm_fft_c2r(acm_ctx* c, int fp64, int nbatch, const void* in, void* out) {
  return fft_impl(c, fp64, nbatch, in, out, false);
}

acm_status acm_history(acm_ctx* c, int index, double* out, int cap, int* count, int* record_len) {
  if (!c || index < 0 || index >= BMAX || cap < 0 || (cap > 0 && !out)) return ACM_ERR_ARG;
  const int len = c->hist_kind == 2 ? SOLUTE_HIST : STOKES_HIST;
  const int n = c->hist_kind == 0 ? 0 : std::min(cap, c->hist_n[index]);
  if (record_len) *record_len = c->hist_kind == 0 ? 0 : len;
  if (count) *count = c->hist_kind == 0 ? 0 : c->hist_n[index];
  if (n > 0) {
    if (c->st) CK(cudaStreamSynchronize(c->st));
    CK(cudaMemcpy(out, c->hist + (size_t)index * HIST_CAP * len, (size_t)n * len * sizeof(double),
                  cudaMemcpyDeviceToHost));
  }
  return ACM_OK;
}

acm_status acm_profile_enable(acm_ctx* c, int on) {
  if (!c) return ACM_ERR_ARG;
  c->prof = on != 0;
  return ACM_OK;
}

acm_status acm_profile_read(acm_ctx* c, double* ms, long long* launches) {
  if (!c) return ACM_ERR_ARG;
  if (c->st) CK(cudaStreamSynchronize(c->st));
  else CK(cudaDeviceSynchronize());
  if (ms) {
    for (int k = 0; k < ACM_K_COUNT; ++k) ms[k] = 0.0;
    for (auto& r : c->recs) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, c->ev[r.second], c->ev[r.second + 1]) == cudaSuccess) ms[r.first] += t;
      else cudaGetLastError();
    }
  }
  if (launches)
    for (int k = 0; k < ACM_K_COUNT; ++k) launches[k] = c->launches[k];
  for (int k = 0; k < ACM_K_COUNT; ++k) c->launches[k] = 0;
  c->recs.clear();
  c->ev_used = 0;
  return ACM_OK;
}

acm_status acm_batch_create(acm_batch** out, int ncells, const int* dims, void* stream) {
  if (!out || ncells < 1 || !dims) return ACM_ERR_ARG;
  *out = nullptr;
  acm_batch* b = new (std::nothrow) acm_batch();
  if (!b) return ACM_ERR_NOMEM;
  b->st = (cudaStream_t)stream;
  b->ncells = ncells;
  for (int i = 0; i < ncells; ++i) {
    const int* d = dims + 3 * i;
    if (!shape_ok(d[0], d[1], d[2])) {
      delete b;
      return ACM_ERR_UNSUPPORTED_SIZE;
    }
    BatchGroup* gr = nullptr;
    for (auto& x : b->groups)
      if (x.n[0] == d[0] && x.n[1] == d[1] && x.n[2] == d[2]) gr = &x;
    if (!gr) {
      b->groups.push_back(BatchGroup());
      gr = &b->groups.back();
      gr->n[0] = d[0];
      gr->n[1] = d[1];
      gr->n[2] = d[2];
    }
    gr->cells.push_back(i);
  }
  acm_status s = ACM_OK;
  for (auto& gr : b->groups) {
    s = ctx_create(&gr.c, gr.n[0], gr.n[1], gr.n[2], stream, 3 * (int)gr.cells.size(), (int)gr.cells.size());
    if (s != ACM_OK) break;
    gr.c->spec_comps = 3;  // Stokes only
  }
  if (s == ACM_OK && (cudaMalloc(&b->counts, (size_t)2 * ncells * sizeof(unsigned long long)) != cudaSuccess ||
                      cudaMalloc(&b->graph.counter, sizeof(unsigned int)) != cudaSuccess)) {
    cudaGetLastError();
    s = ACM_ERR_NOMEM;
  }
  if (s != ACM_OK) {
    acm_batch_destroy(b);
    return s;
  }
  *out = b;
  return ACM_OK;
}

acm_status acm_batch_destroy(acm_batch* b) {
  if (!b) return ACM_ERR_ARG;
  if (b->st) cudaStreamSynchronize(b->st);
  else cudaDeviceSynchronize();
  for (auto& gr : b->groups)
    if (gr.c) acm_destroy(gr.c);
  if (b->graph.exec) cudaGraphExecDestroy(b->graph.exec);
  if (b->graph.counter) cudaFree(b->graph.counter);
  if (b->counts) cudaFree(b->counts);
  cudaGetLastError();
  delete b;
  return ACM_OK;
}

acm_status acm_batch_stokes(acm_batch* b, const uint8_t* const* H, const acm_stokes_params* prm,
                            const void* const* init_u, const void* const* init_lambda, void* const* u_out,
                            void* const* lambda_out, double* K, acm_report* rep) {
  if (!b || !H || !K) return ACM_ERR_ARG;
  acm_stokes_params P;
  fill_stokes_params(prm, &P);
  CKS(check_stokes_args(P));
  if (P.precision == ACM_FP32_THEN_FP64) return ACM_ERR_ARG;
  return P.precision == ACM_FP32 ? batch_stokes_run<float>(b, H, P, init_u, init_lambda, u_out, lambda_out, K, rep)
                                 : batch_stokes_run<double>(b, H, P, init_u, init_lambda, u_out, lambda_out, K, rep);
}

acm_status acm_batch_profile_read(acm_batch* b, double* ms, long long* launches) {
  if (!b) return ACM_ERR_ARG;
  double acc[ACM_K_COUNT] = {};
  long long cnt[ACM_K_COUNT] = {};
  for (auto& gr : b->groups) {
    double m[ACM_K_COUNT];
    long long n[ACM_K_COUNT];
    CKS(acm_profile_read(gr.c, m, n));
    for (int k = 0; k < ACM_K_COUNT; ++k) {
      acc[k] += m[k];
      cnt[k] += n[k];
    }
  }
  for (int k = 0; k < ACM_K_COUNT; ++k) {
    if (ms) ms[k] = acc[k];
    if (launches) launches[k] = cnt[k];
  }
  return ACM_OK;
}

acm_status acm_autotune(acm_ctx* c, int fp64, int deriv, int tiles[NTUNE]) {
  if (!c || (fp64 != 0 && fp64 != 1) || (deriv != 0 && deriv != 1)) return ACM_ERR_ARG;
  CKS(fp64 ? autotune_ctx<double>(c, c->B, deriv) : autotune_ctx<float>(c, c->B, deriv));
  if (tiles) tiles_of(c, fp64, tiles);
  return ACM_OK;
}

acm_status acm_set_tiles(acm_ctx* c, int fp64, const int tiles[NTUNE]) {
  if (!c || !tiles || (fp64 != 0 && fp64 != 1)) return ACM_ERR_ARG;
  Geo g = c->g;
  for (int i = 0; i < NTUNE; ++i) {
    const TuneJob& j = TUNE_JOBS[i];
    if (j.solute && c->spec_comps < 4) continue;
    const int n = j.axis == 1 ? g.n1 : g.n0;
    bool found = false;
    for (int sh = -1; sh <= 4 && !found; ++sh) {
      if (!(fp64 ? Ops<double>::tx_variant(n, j.op, j.nc, sh) : Ops<float>::tx_variant(n, j.op, j.nc, sh))) continue;
      g.txs[fp64][j.axis][j.op] = (signed char)sh;
      const int tx = fp64 ? Ops<double>::pass_tx(g, j.axis, j.op, j.nc) : Ops<float>::pass_tx(g, j.axis, j.op, j.nc);
      found = tx == tiles[i];
    }
    if (!found) return ACM_ERR_ARG;
  }
  c->g = g;
  drop_graphs(c);
  return ACM_OK;
}

acm_status acm_get_tiles(acm_ctx* c, int fp64, int tiles[NTUNE]) {
  if (!c || !tiles || (fp64 != 0 && fp64 != 1)) return ACM_ERR_ARG;
  tiles_of(c, fp64, tiles);
  return ACM_OK;
}

acm_status acm_batch_autotune(acm_batch* b, int fp64, int deriv) {
  if (!b || (fp64 != 0 && fp64 != 1) || (deriv != 0 && deriv != 1)) return ACM_ERR_ARG;
  for (auto& gr : b->groups) {
    const int np = 3 * (int)gr.cells.size();
    CKS(fp64 ? autotune_ctx<double>(gr.c, np, deriv) : autotune_ctx<float>(gr.c, np, deriv));
  }
  if (b->graph.exec) {
    cudaGraphExecDestroy(b->graph.exec);
    b->graph.exec = nullptr;
  }
  return ACM_OK;
}

acm_status acm_batch_tiles(acm_batch* b, int cell, int fp64, int tiles[NTUNE]) {
  if (!b || !tiles || cell < 0 || cell >= b->ncells || (fp64 != 0 && fp64 != 1)) return ACM_ERR_ARG;
  for (auto& gr : b->groups)
    for (int c : gr.cells)
      if (c == cell) {
        tiles_of(gr.c, fp64, tiles);
        return ACM_OK;
      }
  return ACM_ERR_ARG;
}

acm_status acm_batch_history_enable(acm_batch* b, int cap) {
  if (!b || cap < 0) return ACM_ERR_ARG;
  if (b->st) CK(cudaStreamSynchronize(b->st));
  for (auto& gr : b->groups) {
    acm_ctx* c = gr.c;
    if (c->hist_b) cudaFree(c->hist_b);
    c->hist_b = nullptr;
    c->hist_b_cap = 0;
    if (cap > 0) {
      if (cudaMalloc(&c->hist_b, (size_t)c->B * cap * STOKES_HIST * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return ACM_ERR_NOMEM;
      }
      c->hist_b_cap = cap;
    }
    gr.iters.clear();
  }
  // a captured loop holds the old history pointer
  if (b->graph.exec) {
    cudaGraphExecDestroy(b->graph.exec);
    b->graph.exec = nullptr;
  }
  return ACM_OK;
}

acm_status acm_batch_history(acm_batch* b, int cell, int load, double* out, int cap, int* count) {
  if (!b || cell < 0 || cell >= b->ncells || load < 0 || load > 2 || cap < 0 || (cap > 0 && !out))
    return ACM_ERR_ARG;
  for (auto& gr : b->groups) {
    for (size_t i = 0; i < gr.cells.size(); ++i) {
      if (gr.cells[i] != cell) continue;
      acm_ctx* c = gr.c;
      const int p = 3 * (int)i + load;
      const int recorded = c->hist_b && !gr.iters.empty() ? std::min(gr.iters[p], c->hist_b_cap) : 0;
      if (count) *count = recorded;
      const int n = std::min(cap, recorded);
      if (n > 0)
        CK(cudaMemcpy(out, c->hist_b + (size_t)p * c->hist_b_cap * STOKES_HIST, (size_t)n * STOKES_HIST * sizeof(double),
                      cudaMemcpyDeviceToHost));
      return ACM_OK;
    }
  }
  return ACM_ERR_ARG;
}

acm_status acm_batch_profile_enable(acm_batch* b, int on) {
  if (!b) return ACM_ERR_ARG;
  for (auto& gr : b->groups) acm_profile_enable(gr.c, on);
  return ACM_OK;
}

const char* acm_last_error(void) { return g_last_error; }

const char* acm_status_str(acm_status s) {
  switch (s) {
    case ACM_OK: return "ok";
    case ACM_ERR_ARG: return "invalid argument";
    case ACM_ERR_NOMEM: return "device allocation failed";
    case ACM_ERR_CUDA: return "CUDA runtime error";
    case ACM_ERR_MAXITER: return "iteration cap reached before the tolerance";
    case ACM_ERR_DIVERGED: return "iteration diverged";
    case ACM_ERR_NONFINITE: return "non-finite residual";
    case ACM_ERR_NO_SOLID: return "indicator has no solid voxel";
    case ACM_ERR_NO_FLUID: return "indicator has no pore voxel";
    case ACM_ERR_TIMEOUT: return "bounded device wait timed out";
    case ACM_ERR_UNSUPPORTED_SIZE: return "unsupported grid size";
  }
  return "unknown status";
}

}  // extern "C"
