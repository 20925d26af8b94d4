// C ABI of the lgw library: argument checks, host/device staging, workspace
// management and the per-sub-batch schedule of the hot path.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "lgw_internal.cuh"

using namespace lgw;

struct lgw_handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  lgw_status last = LGW_OK;
  std::string msg;
  unsigned *d_status = nullptr;
  struct Buf {
    void *p = nullptr;
    size_t n = 0;
  };
  std::map<std::string, Buf> bufs;
  size_t ws_limit = 0;   // bytes the workspace may hold (0: no limit)
  size_t ws_bytes = 0;   // bytes it holds
  int launches = 0;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  bool timing = false;
  // captured sub-batch graphs; ws_gen changes whenever a workspace buffer is
  // (re)allocated, which also drops every cached graph
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
  };
  std::map<std::string, Graph> graphs;
  unsigned long long ws_gen = 0;
  cudaStream_t cap_stream = nullptr;   // private non-blocking stream for captures
  // lgw_sigma_c_batched runs systems concurrently on these streams, each
  // with its own workspace namespace (ws_prefix)
  std::vector<cudaStream_t> lanes;
  std::string ws_prefix;
  void drop_graphs() {
    for (auto &kv : graphs)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    graphs.clear();
  }
};

struct lgw_system {
  lgw_handle *h = nullptr;
  SysDev s{};
  // spectral interval of C for the polynomial form, estimated on first use
  bool ivl_ok = false;
  double ivl_lo = 0.0, ivl_hi = 0.0;
  __nv_bfloat16 *Ltb_lo = nullptr;   // bf16(L - bf16(L))^T [A][N], made on first use
  // Tamm-Dancoff view (A = Delta + (c_K/2) L L^T in place of C), made on first use
  SysDev tda{};
  void *tda_buf = nullptr;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
namespace {

struct Fail {
  lgw_status st;
};

lgw_status set_err(lgw_handle *h, lgw_status st, const char *fmt, ...) {
  if (h) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    h->last = st;
    h->msg = buf;
  }
  return st;
}

#define LGW_TRY_CUDA(h, call)                                                             \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      set_err((h), e_ == cudaErrorMemoryAllocation ? LGW_ERR_OOM : LGW_ERR_CUDA,          \
              "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      throw Fail{(h)->last};                                                              \
    }                                                                                     \
  } while (0)

void check_launch(lgw_handle *h, const char *what) {
  h->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_err(h, LGW_ERR_CUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
    throw Fail{h->last};
  }
}

void *ws(lgw_handle *h, const std::string &name, size_t bytes) {
  auto &b = h->bufs[h->ws_prefix + name];
  if (bytes == 0) bytes = 8;
  if (b.n < bytes) {
    // the handle's byte limit is checked before anything is freed, so a
    // refused request leaves the workspace as it was
    if (h->ws_limit && h->ws_bytes - b.n + bytes > h->ws_limit) {
      set_err(h, LGW_ERR_OOM,
              "workspace limit: %s needs %zu bytes, the handle holds %zu of its %zu-byte limit",
              name.c_str(), bytes, h->ws_bytes, h->ws_limit);
      throw Fail{LGW_ERR_OOM};
    }
    if (b.p) {
      LGW_TRY_CUDA(h, cudaStreamSynchronize(h->stream));
      cudaFree(b.p);
      h->ws_bytes -= b.n;
      b.p = nullptr;
      b.n = 0;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_err(h, LGW_ERR_OOM, "cudaMalloc(%zu bytes) for %s failed: %s", bytes, name.c_str(),
              cudaGetErrorString(e));
      throw Fail{LGW_ERR_OOM};
    }
    b.p = p;
    b.n = bytes;
    h->ws_bytes += bytes;
    h->ws_gen++;
    h->drop_graphs();
  }
  return b.p;
}

template <class T>
T *wsT(lgw_handle *h, const std::string &name, size_t count) {
  return static_cast<T *>(ws(h, name, count * sizeof(T)));
}

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device view of an input: the pointer itself, or a staged copy.
template <class T>
const T *in_dev(lgw_handle *h, const std::string &name, const T *p, size_t count) {
  if (!p || count == 0) return p;
  if (is_device_ptr(p)) return p;
  T *d = wsT<T>(h, name, count);
  LGW_TRY_CUDA(h, cudaMemcpyAsync(d, p, count * sizeof(T), cudaMemcpyHostToDevice, h->stream));
  return d;
}

// Host copy of a small array given on either side.
template <class T>
std::vector<T> to_host(lgw_handle *h, const T *p, size_t count) {
  std::vector<T> v(count);
  if (count == 0) return v;
  if (is_device_ptr(p)) {
    LGW_TRY_CUDA(h, cudaMemcpyAsync(v.data(), p, count * sizeof(T), cudaMemcpyDeviceToHost,
                                    h->stream));
    LGW_TRY_CUDA(h, cudaStreamSynchronize(h->stream));
  } else {
    std::memcpy(v.data(), p, count * sizeof(T));
  }
  return v;
}

// Output staging: compute into a device buffer, copy back if the caller's
// pointer is host memory.
template <class T>
struct OutBuf {
  T *user = nullptr;
  T *dev = nullptr;
  size_t count = 0;
  bool host = false;
  void init(lgw_handle *h, const std::string &name, T *p, size_t n) {
    user = p;
    count = n;
    if (!p) {
      dev = nullptr;
      return;
    }
    host = !is_device_ptr(p);
    dev = host ? wsT<T>(h, name, n) : p;
  }
  void finish(lgw_handle *h) {
    if (user && host && count)
      LGW_TRY_CUDA(h, cudaMemcpyAsync(user, dev, count * sizeof(T), cudaMemcpyDeviceToHost,
                                      h->stream));
  }
};

struct Timer {
  lgw_handle *h;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> spans;
  cudaEvent_t open = nullptr;
  int open_cat = -1;
  explicit Timer(lgw_handle *hh) : h(hh) {}
  cudaEvent_t ev() {
    if (h->ev_used == h->ev_pool.size()) {
      cudaEvent_t e;
      LGW_TRY_CUDA(h, cudaEventCreate(&e));
      h->ev_pool.push_back(e);
    }
    return h->ev_pool[h->ev_used++];
  }
  // Close the running span (if any) and open one for category `cat`.
  void mark(int cat) {
    if (!h->timing) return;
    cudaEvent_t e = ev();
    LGW_TRY_CUDA(h, cudaEventRecord(e, h->stream));
    if (open) spans.push_back({open_cat, {open, e}});
    open = e;
    open_cat = cat;
  }
  void stop() {
    if (!h->timing || !open) return;
    cudaEvent_t e = ev();
    LGW_TRY_CUDA(h, cudaEventRecord(e, h->stream));
    spans.push_back({open_cat, {open, e}});
    open = nullptr;
  }
  void collect(double *acc, int ncat) {
    if (!h->timing) return;
    LGW_TRY_CUDA(h, cudaStreamSynchronize(h->stream));
    for (auto &s : spans) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, s.second.first, s.second.second);
      if (s.first >= 0 && s.first < ncat) acc[s.first] += ms;
    }
    spans.clear();
  }
};

enum Cat { C_START, C_GEMM1, C_GEMM2, C_DOTS, C_UPDATE, C_PASS2, C_NORM, C_SPEC, C_CF, C_QP, C_N };

void check_status(lgw_handle *h) {
  unsigned st = 0;
  LGW_TRY_CUDA(h, cudaMemcpyAsync(&st, h->d_status, sizeof st, cudaMemcpyDeviceToHost, h->stream));
  LGW_TRY_CUDA(h, cudaStreamSynchronize(h->stream));
  if (st & ST_TIMEOUT) {
    set_err(h, LGW_ERR_TIMEOUT, "a bounded device wait ran out");
    throw Fail{LGW_ERR_TIMEOUT};
  }
  if (st & ST_BAD_INPUT) {
    set_err(h, LGW_ERR_SHAPE, "a tridiagonal depth k_eff lies outside [0, k]");
    throw Fail{LGW_ERR_SHAPE};
  }
  if (st & ST_NOT_SPD) {
    set_err(h, LGW_ERR_NOT_SPD, "non-positive pair energy or Gauss node (C not positive definite)");
    throw Fail{LGW_ERR_NOT_SPD};
  }
  if (st & ST_NO_CONV) {
    set_err(h, LGW_ERR_NO_CONVERGENCE, "tridiagonal eigensolver or QP equation did not converge");
    throw Fail{LGW_ERR_NO_CONVERGENCE};
  }
}

// Replay the cached graph for `key`, capturing `body` into it first if it
// is not cached.  A failed capture runs `body` eagerly instead.
template <class F>
void run_graphed(lgw_handle *h, const std::string &key, F &&body) {
  cudaStream_t st = h->stream;
  auto it = h->graphs.find(key);
  if (it == h->graphs.end()) {
    if (h->graphs.size() >= 64) h->drop_graphs();
    // the caller's stream may be the legacy default stream, which cannot be
    // captured: record the launches on the handle's own stream (the graph is
    // then launched on the caller's stream, which orders it)
    if (!h->cap_stream)
      LGW_TRY_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    const int l0 = h->launches;
    LGW_TRY_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaGraph_t g = nullptr;
    h->stream = h->cap_stream;
    try {
      body();
    } catch (Fail &) {
      h->stream = st;
      cudaStreamEndCapture(h->cap_stream, &g);
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      throw;
    }
    h->stream = st;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    cudaGraphExec_t ex = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      h->launches = l0;
      body();
      return;
    }
    lgw_handle::Graph gr;
    gr.exec = ex;
    gr.launches = h->launches - l0;
    h->launches = l0;
    it = h->graphs.emplace(key, gr).first;
  }
  LGW_TRY_CUDA(h, cudaGraphLaunch(it->second.exec, st));
  h->launches += it->second.launches;
}

struct Opts {
  int k, precision, reorth, b_sub, qp_max_iter, use_graph, split, split32, qp_mode;
  double tol, qp_tol;
};

Opts resolve_opts(lgw_handle *h, const lgw_options *o, const SysDev &s) {
  if (!o) {
    set_err(h, LGW_ERR_ARG, "options pointer is NULL");
    throw Fail{LGW_ERR_ARG};
  }
  Opts r;
  r.k = o->k;
  r.precision = o->precision;
  r.reorth = o->reorth;
  r.b_sub = o->b_sub;
  r.qp_max_iter = o->qp_max_iter > 0 ? o->qp_max_iter : 50;
  r.use_graph = o->use_graph;
  r.qp_mode = o->qp_mode;
  if (r.qp_mode != 0 && r.qp_mode != 1) {
    set_err(h, LGW_ERR_ARG, "unknown qp_mode %d", o->qp_mode);
    throw Fail{LGW_ERR_ARG};
  }
  if (o->reorth_arith < LGW_RA_AUTO || o->reorth_arith > LGW_RA_SPLIT32) {
    set_err(h, LGW_ERR_ARG, "unknown reorthogonalisation arithmetic %d", o->reorth_arith);
    throw Fail{LGW_ERR_ARG};
  }
  r.split = o->reorth_arith == LGW_RA_SPLIT || o->reorth_arith == LGW_RA_SPLIT32 ||
            (o->reorth_arith == LGW_RA_AUTO && o->precision != LGW_FP64);
  r.split32 = o->reorth_arith == LGW_RA_SPLIT32;
  r.tol = o->breakdown_tol > 0 ? o->breakdown_tol : 1e-13;
  r.qp_tol = o->qp_tol > 0 ? o->qp_tol : 1e-10;
  if (r.k < 1 || r.k > s.n_vc) {
    set_err(h, LGW_ERR_ARG, "k = %d outside [1, n_vc = %d]", r.k, s.n_vc);
    throw Fail{LGW_ERR_ARG};
  }
  if (r.k > 4095) {
    set_err(h, LGW_ERR_UNSUPPORTED, "k = %d above the 4095-step limit of this build", r.k);
    throw Fail{LGW_ERR_UNSUPPORTED};
  }
  if (r.precision != LGW_FP64 && r.precision != LGW_BF16 && r.precision != LGW_FP8 &&
      r.precision != LGW_FP8_DEQ) {
    set_err(h, LGW_ERR_ARG, "unknown precision %d", r.precision);
    throw Fail{LGW_ERR_ARG};
  }
  if (r.reorth < LGW_REORTH_NONE || r.reorth > LGW_REORTH_DCGS) {
    set_err(h, LGW_ERR_ARG, "unknown reorthogonalisation mode %d", r.reorth);
    throw Fail{LGW_ERR_ARG};
  }
  if (r.b_sub < 0) {
    set_err(h, LGW_ERR_ARG, "b_sub < 0");
    throw Fail{LGW_ERR_ARG};
  }
  if (r.precision != LGW_FP64 && !tc_available()) {
    set_err(h, LGW_ERR_UNSUPPORTED, "tensor-core paths need an sm_103 device");
    throw Fail{LGW_ERR_UNSUPPORTED};
  }
  return r;
}

// E4M3 copies of L from src [nr][nc] (row stride ld) into s.
void make_fp8(lgw_handle *h, SysDev &s, const double *src, int ld, int nr, int nc) {
  const size_t n = (size_t)s.N * s.A;
  uint8_t *a = nullptr, *b = nullptr;
  float *sc = nullptr;
  if (cudaMalloc(&a, n) != cudaSuccess || cudaMalloc(&b, n) != cudaSuccess ||
      cudaMalloc(&sc, sizeof(float) * s.A) != cudaSuccess) {
    cudaGetLastError();
    if (a) cudaFree(a);
    if (b) cudaFree(b);
    if (sc) cudaFree(sc);
    set_err(h, LGW_ERR_OOM, "device allocation for the E4M3 copies of L failed");
    throw Fail{LGW_ERR_OOM};
  }
  unsigned *colmax = wsT<unsigned>(h, "fp8_colmax", (size_t)s.A);
  launch_prepare_fp8(src, ld, nr, nc, s, colmax, a, b, sc, h->stream);
  check_launch(h, "prepare_fp8");
  s.L8 = a;
  s.L8t = b;
  s.sL = sc;
}

// The copies of L a request needs must exist; the E4M3 copies are made on
// the first FP8 request for a system that keeps its FP64 copy.
void ensure_copies(lgw_handle *h, const lgw_system *csys, const Opts &o) {
  const SysDev &cs = csys->s;
  if (o.precision == LGW_FP64 && !cs.L64) {
    set_err(h, LGW_ERR_UNSUPPORTED, "the system keeps no FP64 copy of L (LGW_SYS_NO_FP64)");
    throw Fail{LGW_ERR_UNSUPPORTED};
  }
  if (o.precision == LGW_BF16 && !cs.Lb) {
    set_err(h, LGW_ERR_UNSUPPORTED, "the system keeps no BF16 copy of L (LGW_SYS_NO_BF16)");
    throw Fail{LGW_ERR_UNSUPPORTED};
  }
  if ((o.precision != LGW_FP8 && o.precision != LGW_FP8_DEQ) || cs.L8) return;
  if (!cs.L64) {
    set_err(h, LGW_ERR_UNSUPPORTED, "no E4M3 copy of L and no FP64 copy to make it from");
    throw Fail{LGW_ERR_UNSUPPORTED};
  }
  lgw_system *sys = const_cast<lgw_system *>(csys);
  make_fp8(h, sys->s, cs.L64, cs.A, cs.N, cs.A);
}

struct ProbView {
  int n_t, n_m, n_freq, B;
  std::vector<int> targets, m_idx;
  const int *d_targets, *d_m_idx;
  const double *d_M, *d_V, *d_omega, *d_shift;
  double delta;
};

ProbView check_problem(lgw_handle *h, const SysDev &s, const lgw_problem *p) {
  if (!p) {
    set_err(h, LGW_ERR_ARG, "problem pointer is NULL");
    throw Fail{LGW_ERR_ARG};
  }
  ProbView v{};
  v.n_t = p->n_t;
  v.n_m = p->n_m;
  v.n_freq = p->n_freq;
  if (v.n_t < 0 || v.n_m < 0 || v.n_freq < 0 || (v.n_t > 0 && !p->targets) ||
      (v.n_m > 0 && !p->m_idx) || (v.n_freq > 0 && !p->omega)) {
    set_err(h, LGW_ERR_ARG, "negative size or missing targets/m_idx/omega");
    throw Fail{LGW_ERR_ARG};
  }
  if ((p->M == nullptr) == (p->V == nullptr)) {
    set_err(h, LGW_ERR_ARG, "exactly one of M and V must be given");
    throw Fail{LGW_ERR_ARG};
  }
  if (!(p->delta > 0.0)) {
    set_err(h, LGW_ERR_ARG, "delta must be > 0");
    throw Fail{LGW_ERR_ARG};
  }
  v.B = v.n_t * v.n_m;
  v.targets = to_host(h, p->targets, v.n_t);
  v.m_idx = to_host(h, p->m_idx, v.n_m);
  const int norb = s.n_v + s.n_c;
  for (int t : v.targets)
    if (t < 0 || t >= norb) {
      set_err(h, LGW_ERR_SHAPE, "target index %d outside [0, %d)", t, norb);
      throw Fail{LGW_ERR_SHAPE};
    }
  for (int m : v.m_idx)
    if (m < 0 || m >= norb) {
      set_err(h, LGW_ERR_SHAPE, "summed index %d outside [0, %d)", m, norb);
      throw Fail{LGW_ERR_SHAPE};
    }
  v.d_targets = in_dev(h, "in_targets", v.targets.data(), (size_t)v.n_t);
  v.d_m_idx = in_dev(h, "in_midx", v.m_idx.data(), (size_t)v.n_m);
  v.d_omega = in_dev(h, "in_omega", p->omega, (size_t)v.n_freq);
  v.d_shift = p->static_shift ? in_dev(h, "in_shift", p->static_shift, (size_t)v.n_t) : nullptr;
  v.d_M = p->M ? in_dev(h, "in_M", p->M, (size_t)v.B * s.n_aux) : nullptr;
  v.d_V = p->V ? in_dev(h, "in_V", p->V, (size_t)v.B * s.n_vc) : nullptr;
  v.delta = p->delta;
  return v;
}

// ---------------------------------------------------------------------------
// Lanczos over all start vectors, sub-batch by sub-batch.
// alpha/beta [B][k], beta0 [B], k_eff [B] are device arrays.
// ---------------------------------------------------------------------------
// Polynomial operator D = p_g(C) (the paper's form after Eq. 12): the
// Chebyshev interpolant of sqrt at the g+1 points of the first kind on
// [lo, hi], applied by Clenshaw's recurrence in S = a_s C + b_s I.
struct PolyOp {
  int g;
  double lo, hi, as, bs;
  std::vector<double> c;   // c_0 .. c_g
};

PolyOp make_poly(int g, double lo, double hi) {
  PolyOp p;
  p.g = g;
  p.lo = lo;
  p.hi = hi;
  p.as = 2.0 / (hi - lo);
  p.bs = -(hi + lo) / (hi - lo);
  const int n = g + 1;
  const double pi = 3.14159265358979323846;
  std::vector<double> f(n);
  for (int j = 0; j < n; ++j)
    f[j] = std::sqrt(0.5 * (hi + lo) + 0.5 * (hi - lo) * std::cos(pi * (j + 0.5) / n));
  p.c.assign(n, 0.0);
  for (int k = 0; k < n; ++k) {
    double acc = 0.0;
    for (int j = 0; j < n; ++j) acc += f[j] * std::cos(k * pi * (j + 0.5) / n);
    p.c[k] = 2.0 / n * acc;
  }
  p.c[0] *= 0.5;
  return p;
}

// keep_basis stores all k + 1 FP64 basis vectors of a sub-batch (slot j of
// sub-batch row b at basis + (j * Bs + b) * N) whatever the reorthogonalisation
// mode; after_sub, if given, runs once each sub-batch's recurrence is done.
using SubBatchHook = std::function<void(const VecCtx &)>;
// after_step, if given, runs after the start (j = -1) and after each step j
// that ends with the plain normalisation (FP64 basis or ring; not the split
// basis), once q_{j+1} is in its slot.
using StepHook = std::function<void(const VecCtx &, int)>;

void run_lanczos(lgw_handle *h, const SysDev &s, const ProbView &pv, const Opts &o, double *alpha,
                 double *beta, double *beta0, int *k_eff, lgw_report *rep, double *tacc,
                 bool keep_basis = false, const SubBatchHook *after_sub = nullptr,
                 const PolyOp *poly = nullptr, const StepHook *after_step = nullptr) {
  // a reference: a graph capture redirects the launches to the capture stream
  cudaStream_t &st = h->stream;
  const int B = pv.B;
  const int k = o.k;
  if (B == 0) return;
  LGW_TRY_CUDA(h, cudaMemsetAsync(alpha, 0, sizeof(double) * B * k, st));
  LGW_TRY_CUDA(h, cudaMemsetAsync(beta, 0, sizeof(double) * B * k, st));
  const bool tc = o.precision != LGW_FP64;
  const bool fp8 = o.precision == LGW_FP8;
  const bool deq = o.precision == LGW_FP8_DEQ;
  int nsub_req = o.b_sub > 0 ? o.b_sub : std::min(B, 512);
  nsub_req = std::min(nsub_req, B);
  int Bs = round_up(nsub_req, PAD_VEC);
  if (tc) Bs = std::max(Bs, 64);
  const int N = s.N;
  const int nchunks = (N + VEC_CHUNK - 1) / VEC_CHUNK;
  const int kmax1 = k + 1;
  const bool reorth = o.reorth != LGW_REORTH_NONE;
  const bool split = reorth && o.split;
  // the delayed single-sweep Gram-Schmidt runs on the split basis; with the
  // FP64 basis the same request runs as CGS1K
  const bool dcgs = split && o.reorth == LGW_REORTH_DCGS;
  const bool full_basis = !split && (reorth || keep_basis);
  const int nslots = full_basis ? k + 1 : 3;

  VecCtx c{};
  c.N = N;
  c.Bs = Bs;
  c.nchunks = nchunks;
  c.k = k;
  c.kmax1 = kmax1;
  c.reorth = (o.reorth == LGW_REORTH_DCGS && !dcgs) ? (int)LGW_REORTH_CGS1K : o.reorth;
  c.ring = full_basis ? 0 : 1;
  c.nslots = nslots;
  c.tol = o.tol;
  c.Delta2 = s.Delta2;
  c.dsq = s.dsq;
  c.cd = s.cd;
  c.w = wsT<double>(h, "w", (size_t)Bs * N);
  c.basis = wsT<double>(h, split ? "ring" : "basis", (size_t)nslots * Bs * N);
  if (split) {
    c.bhi = wsT<float>(h, "basis_hi", (size_t)(k + 1) * Bs * N);
    c.blo = o.split32 ? nullptr : wsT<float>(h, "basis_lo", (size_t)(k + 1) * Bs * N);
  }
  c.dsqf = s.dsqf;
  c.d2lo = s.d2lo;
  // tensor cores without reorthogonalisation (the three-vector ring): the
  // slots and w as float pairs, the vector passes in double-float arithmetic
  c.pair = (tc && !reorth && !full_basis && poly == nullptr && s.d2lo != nullptr) ? 1 : 0;
  c.nalpha_f = c.pair ? wsT<float2>(h, "nalpha_f", (size_t)Bs) : nullptr;
  c.nbeta_f = c.pair ? wsT<float2>(h, "nbeta_f", (size_t)Bs) : nullptr;
  // float [Bs][N]: the split-basis epilogue output (c_K Delta^1/2 U) and, at
  // the start of each sub-batch, the tensor-core coupling vectors V = L M
  float *ucd_buf = tc ? wsT<float>(h, "ucd", (size_t)Bs * N) : nullptr;
  c.ucd = split ? ucd_buf : nullptr;
  c.d2f = s.d2f;
  c.kf = s.kf;
  c.n_yb = (s.A + 255) / 256;
  float *yy = (split && tc) ? wsT<float>(h, "yy_part", (size_t)Bs * c.n_yb) : nullptr;
  c.yy_part = yy;
  // the delayed sweep reads step j's partials and writes step j + 1's in
  // the same launch: two halves by step parity (the start writes half 0)
  c.dq2_part = (split && tc) ? wsT<float>(h, "dq2_part", (size_t)(dcgs ? 2 : 1) * Bs * nchunks)
                             : nullptr;
  c.xh = tc ? wsT<__nv_bfloat16>(h, "xh", (size_t)Bs * N) : nullptr;
  // alpha partials: per 2048-element chunk (tensor cores without
  // reorthogonalisation), per GEMM2 tile otherwise
  const bool tc_plain = tc && !reorth;
  c.n_mt = (tc_plain || poly) ? nchunks : (tc ? tc_n_mt(s) : N / F64_TILE);
  // chunks per block of the assembly, axpy and normalisation passes on the
  // tensor-core path without reorthogonalisation; 1 unless LGW_VEC_CPB (1 to
  // 64) asks otherwise (2, 4 and 8 measured within 3% of 1, bit-identical)
  c.cpb = 1;
  if (tc_plain) {
    if (const char *env = std::getenv("LGW_VEC_CPB"))
      c.cpb = std::max(1, std::min(64, std::atoi(env)));
  }
  c.alpha_part = wsT<double>(h, "alpha_part", (size_t)c.n_mt * Bs);
  c.dot_part = reorth ? wsT<double>(h, "dot_part", (size_t)Bs * nchunks * kmax1) : nullptr;
  c.h = reorth ? wsT<double>(h, "hcoef", (size_t)Bs * kmax1) : nullptr;
  c.norm_a = wsT<double>(h, "norm_a", (size_t)Bs * nchunks);
  c.norm_b = wsT<double>(h, "norm_b", (size_t)Bs * nchunks);
  c.norm_c = wsT<double>(h, "norm_c", (size_t)Bs * nchunks);
  c.flag2 = wsT<int>(h, "flag2", (size_t)Bs);
  c.amax = wsT<double>(h, "amax", (size_t)Bs);
  c.betaj = wsT<double>(h, "betaj", (size_t)Bs);
  c.sinv = wsT<double>(h, "sinv", (size_t)Bs);
  c.alpha = alpha;
  c.beta = beta;
  c.beta0 = beta0;
  c.k_eff = k_eff;
  c.n_second = wsT<int>(h, "n_second", 1);
  c.status = h->d_status;
  if (dcgs) {
    // the carried vector lives in ring slot 0 (where the start writes q_0);
    // FP64 contractions leave C w in the w buffer
    c.wv = slot_ptr(c, 0);
    c.uC = tc ? nullptr : c.w;
    c.hj_part = wsT<double>(h, "hj_part", (size_t)Bs * nchunks);
    c.gq = wsT<double>(h, "gq", (size_t)Bs * kmax1);
  }
  LGW_TRY_CUDA(h, cudaMemsetAsync(c.n_second, 0, sizeof(int), st));
  LGW_TRY_CUDA(h, cudaMemsetAsync(c.flag2, 0, sizeof(int) * Bs, st));

  // contraction buffers
  double *Y64 = wsT<double>(h, "y64", (size_t)Bs * s.A);
  const int splits64 = gemm1_f64_splits(s, Bs);
  double *Yp64 = tc ? nullptr : wsT<double>(h, "yp64", (size_t)splits64 * Bs * s.A);
  TcPlan *plan = nullptr;
  uint8_t *x8 = nullptr, *y8 = nullptr;
  uint16_t *x16 = nullptr, *y16 = nullptr;
  float *sx = nullptr, *ty = nullptr;
  float *Yp32 = nullptr;
  __nv_bfloat16 *Yh = nullptr;
  int splits_tc = 1;
  if (tc) {
    // the split count only depends on shapes; size the partials generously
    Yp32 = wsT<float>(h, "yp32", (size_t)64 * Bs * s.A);
    Yh = wsT<__nv_bfloat16>(h, "yh", (size_t)Bs * s.A);
    char err[256];
    plan = tc_plan_create(s, Bs, c.xh, Yp32, Yh, &splits_tc, err, sizeof err);
    if (!plan) {
      set_err(h, LGW_ERR_CUDA, "%s", err);
      throw Fail{LGW_ERR_CUDA};
    }
    if (!fp8 && !deq && !tc_plan_has_bf16(plan)) {
      tc_plan_destroy(plan);
      set_err(h, LGW_ERR_UNSUPPORTED, "BF16 contractions need the BF16 copies of L");
      throw Fail{LGW_ERR_UNSUPPORTED};
    }
    if (deq) {
      x16 = wsT<uint16_t>(h, "x16", (size_t)Bs * N);
      y16 = wsT<uint16_t>(h, "y16", (size_t)Bs * s.A);
      sx = wsT<float>(h, "sx", (size_t)Bs);
      ty = wsT<float>(h, "ty", (size_t)Bs);
      if (!tc_plan_enable_deq(plan, s.L8t, s.L8, x16, y16, ty)) {
        tc_plan_destroy(plan);
        set_err(h, LGW_ERR_CUDA, "cuTensorMapEncodeTiled failed for the widened E4M3 operands");
        throw Fail{LGW_ERR_CUDA};
      }
    }
    if (fp8) {
      x8 = wsT<uint8_t>(h, "x8", (size_t)Bs * N);
      y8 = wsT<uint8_t>(h, "y8", (size_t)Bs * s.A);
      sx = wsT<float>(h, "sx", (size_t)Bs);
      ty = wsT<float>(h, "ty", (size_t)Bs);
      if (!tc_plan_enable_fp8(plan, s.L8t, s.L8, x8, y8, ty)) {
        tc_plan_destroy(plan);
        set_err(h, LGW_ERR_CUDA, "cuTensorMapEncodeTiled failed for the E4M3 operands");
        throw Fail{LGW_ERR_CUDA};
      }
    }
    if (!tc_plan_autotune(plan, ucd_buf, h->d_status, st, &splits_tc)) {
      tc_plan_destroy(plan);
      set_err(h, LGW_ERR_CUDA, "tensor-core tile autotuning failed");
      throw Fail{LGW_ERR_CUDA};
    }
  }
  struct PlanGuard {
    TcPlan *p;
    ~PlanGuard() {
      if (p) tc_plan_destroy(p);
    }
  } guard{plan};

  // use_graph: each sub-batch's launch sequence (start vectors and the k
  // steps) is captured once and replayed from the handle's graph cache
  const bool graph_mode = o.use_graph && after_sub == nullptr;
  const bool timing_saved = h->timing;
  if (graph_mode) h->timing = false;
  struct TimingRestore {
    lgw_handle *h;
    bool v;
    ~TimingRestore() { h->timing = v; }
  } timing_restore{h, timing_saved};
  // Clenshaw buffers of the polynomial operator
  double *pb[3] = {nullptr, nullptr, nullptr};
  double *pT = nullptr;
  if (poly) {
    for (int i = 0; i < 3; ++i)
      pb[i] = wsT<double>(h, "poly_b" + std::to_string(i), (size_t)Bs * N);
    if (!tc) pT = wsT<double>(h, "poly_t", (size_t)Bs * N);
  }
  // C b for the polynomial operator: FP64 product into pT, or the tensor
  // cores from c.xh = bf16(Delta^1/2 b) into ucd_buf
  auto apply_c = [&](const double *bsrc) {
    if (tc) {
      if (fp8) {
        launch_quant_x8(c.xh, Bs, N, x8, sx, st);
        check_launch(h, "quant_x8");
      } else if (deq) {
        launch_quant_x16(c.xh, Bs, N, x16, sx, st);
        check_launch(h, "quant_x16");
      }
      launch_gemm1_tc(plan, h->d_status, st);
      check_launch(h, "gemm1_tc");
      if (fp8)
        launch_reduce_y_fp8(Yp32, splits_tc, Bs, s.A, sx, s.sL, y8, ty, nullptr, 1, st);
      else if (deq)
        launch_reduce_y_f16(Yp32, splits_tc, Bs, s.A, sx, s.sL, y16, ty, nullptr, 1, st);
      else
        launch_reduce_y_bf16(Yp32, splits_tc, Bs, s.A, Yh, nullptr, st);
      check_launch(h, "reduce_y");
      launch_gemm2_tc_split(plan, ucd_buf, h->d_status, st);
      check_launch(h, "gemm2_tc");
    } else {
      launch_gemm1_f64(s, bsrc, Bs, Yp64, splits64, st);
      check_launch(h, "gemm1_f64");
      launch_reduce_y_f64(Yp64, splits64, Bs, s.A, Y64, st);
      check_launch(h, "reduce_y_f64");
      launch_gemm2_f64(s, Y64, Bs, EPI_APPLY, bsrc, nullptr, nullptr, pT, nullptr, st);
      check_launch(h, "gemm2_f64");
    }
  };
  Timer tm(h);
  int nsub = 0;
  for (int vec0 = 0; vec0 < B; vec0 += nsub_req, ++nsub) {
    const int nvec = std::min(nsub_req, B - vec0);
    c.vec0 = vec0;
    c.nvec = nvec;
    auto sub_body = [&]() {
      // ---- start vectors b = Delta^1/2 V, V = L M (text after Eq. 8) ----
      tm.mark(C_START);
      if (pv.d_M && tc && s.Lb) {
        // V = L M on the tensor cores in split BF16 (three products, FP32 sum)
        float *vf = ucd_buf;
        if (!launch_coupling_tc(plan, s, pv.d_M + (size_t)vec0 * s.n_aux, nvec, vf, h->d_status,
                                st)) {
          set_err(h, LGW_ERR_UNSUPPORTED, "tensor-core plan without the BF16 copies of L");
          throw Fail{LGW_ERR_UNSUPPORTED};
        }
        check_launch(h, "coupling_tc");
        launch_start_from_vf(c, vf, st);
        check_launch(h, "start_from_vf");
      } else if (pv.d_M) {
        if (!s.L64) {
          set_err(h, LGW_ERR_UNSUPPORTED, "start vectors from M need the BF16 or FP64 copy of L");
          throw Fail{LGW_ERR_UNSUPPORTED};
        }
        LGW_TRY_CUDA(h, cudaMemsetAsync(Y64, 0, sizeof(double) * Bs * s.A, st));
        LGW_TRY_CUDA(h, cudaMemcpy2DAsync(Y64, sizeof(double) * s.A, pv.d_M + (size_t)vec0 * s.n_aux,
                                          sizeof(double) * s.n_aux, sizeof(double) * s.n_aux, nvec,
                                          cudaMemcpyDeviceToDevice, st));
        launch_gemm2_f64(s, Y64, Bs, EPI_START, nullptr, nullptr, nullptr, c.w, nullptr, st);
        check_launch(h, "gemm2_f64(start)");
        // padding rows of w (b >= nvec) hold L*0 = 0 already
        launch_norm_partials(c, c.w, c.norm_a, st);
        check_launch(h, "norm_partials");
      } else {
        launch_start_from_v(c, pv.d_V + (size_t)vec0 * s.n_vc, s.n_vc, s.n_vc, st);
        check_launch(h, "start_from_v");
      }
      if (split)
        launch_start_split(c, st);
      else
        launch_normalize(c, 0, 1, nullptr, st);
      check_launch(h, "normalize(start)");
      if (after_step) (*after_step)(c, -1);

      for (int j = 0; j < k; ++j) {
        const double *qj = slot_ptr(c, j);
        const double *qp = j > 0 ? slot_ptr(c, j - 1) : nullptr;
        // ---- C q_j through the two contractions (Eq. 4) ----
        tm.mark(C_GEMM1);
        if (poly) {
          // D q_j = p_g(C) q_j by Clenshaw; w = D q_j - beta_j q_{j-1}
          PolyStep ps{};
          ps.N = N;
          ps.q = qj;
          ps.Delta2 = s.Delta2;
          ps.dsqf = s.dsqf;
          ps.as = poly->as;
          ps.bs = poly->bs;
          ps.xh = tc ? c.xh : nullptr;
          ps.ck = poly->c[poly->g];
          ps.out = pb[0];
          tm.mark(C_UPDATE);
          launch_cheb_step(ps, nchunks, Bs, st);
          check_launch(h, "cheb_step");
          int i1 = 0, i2 = -1;
          for (int kk = poly->g - 1; kk >= 0; --kk) {
            tm.mark(C_GEMM1);
            apply_c(pb[i1]);
            tm.mark(C_UPDATE);
            ps.b1 = pb[i1];
            ps.b2 = i2 >= 0 ? pb[i2] : nullptr;
            ps.T = tc ? nullptr : pT;
            ps.ucd = tc ? ucd_buf : nullptr;
            ps.ck = poly->c[kk];
            if (kk > 0) {
              const int io = (i1 + 1) % 3;
              ps.out = pb[io];
              launch_cheb_step(ps, nchunks, Bs, st);
              check_launch(h, "cheb_step");
              i2 = i1;
              i1 = io;
            } else {
              ps.out = nullptr;
              ps.xh = nullptr;
              launch_cheb_final(ps, qp, c.betaj, c.w, c.alpha_part, nchunks, Bs, st);
              check_launch(h, "cheb_final");
            }
          }
        } else if (tc) {
          // the delayed Gram-Schmidt contracts the unnormalised carried
          // vector; 1/beta_j is applied to each column of the reduction
          const double *vscale = dcgs ? c.sinv : nullptr;
          if (fp8) {
            launch_quant_x8(c.xh, Bs, N, x8, sx, st, vscale);
            check_launch(h, "quant_x8");
          } else if (deq) {
            launch_quant_x16(c.xh, Bs, N, x16, sx, st, vscale);
            check_launch(h, "quant_x16");
          }
          launch_gemm1_tc(plan, h->d_status, st);
          check_launch(h, "gemm1_tc");
          if (fp8)
            launch_reduce_y_fp8(Yp32, splits_tc, Bs, s.A, sx, s.sL, y8, ty, yy, c.n_yb, st);
          else if (deq)
            launch_reduce_y_f16(Yp32, splits_tc, Bs, s.A, sx, s.sL, y16, ty, yy, c.n_yb, st);
          else
            launch_reduce_y_bf16(Yp32, splits_tc, Bs, s.A, Yh, yy, st, vscale);
          check_launch(h, "reduce_y");
          tm.mark(C_GEMM2);
          if (split) {
            launch_gemm2_tc_split(plan, const_cast<float *>(c.ucd), h->d_status, st);
          } else if (tc_plain) {
            // store-only FP32 epilogue; w and the alpha partials in FP64 on
            // the vector pass (an FP64 epilogue would serialise behind the
            // MMAs on the narrow FP64 pipe)
            launch_gemm2_tc_split(plan, ucd_buf, h->d_status, st);
            check_launch(h, "gemm2_tc");
            launch_assemble_w(c, j, ucd_buf, st);
          } else {
            launch_gemm2_tc(plan, EPI_LANCZOS, qj, qp, c.betaj, c.w, c.alpha_part, h->d_status,
                            st);
          }
          check_launch(h, tc_plain ? "assemble_w" : "gemm2_tc");
        } else if (dcgs) {
          // C w_{j-1} in FP64 with the partials of w . C w (alpha~ after
          // scaling by 1/beta_j^2)
          launch_gemm1_f64(s, c.wv, Bs, Yp64, splits64, st);
          check_launch(h, "gemm1_f64");
          launch_reduce_y_f64(Yp64, splits64, Bs, s.A, Y64, st);
          check_launch(h, "reduce_y_f64");
          tm.mark(C_GEMM2);
          launch_gemm2_f64(s, Y64, Bs, EPI_APPLY, c.wv, nullptr, nullptr, c.w, c.alpha_part, st);
          check_launch(h, "gemm2_f64");
        } else {
          launch_gemm1_f64(s, qj, Bs, Yp64, splits64, st);
          check_launch(h, "gemm1_f64");
          launch_reduce_y_f64(Yp64, splits64, Bs, s.A, Y64, st);
          check_launch(h, "reduce_y_f64");
          tm.mark(C_GEMM2);
          launch_gemm2_f64(s, Y64, Bs, EPI_LANCZOS, qj, qp, c.betaj, c.w, c.alpha_part, st);
          check_launch(h, "gemm2_f64");
        }
        // ---- recurrence and reorthogonalisation ----
        tm.mark(C_DOTS);
        if (dcgs) {
          // one sweep over the basis: delayed update of q_j, w_j and its
          // projection coefficients; then beta_{j+1}, and the rare second pass
          launch_sweep_dcgs(c, j, st);
          check_launch(h, "sweep_dcgs");
          tm.mark(C_UPDATE);
          launch_reduce_dcgs(c, j, st);
          check_launch(h, "reduce_dcgs");
          tm.mark(C_PASS2);
          launch_pass2_dcgs(c, j, st);
          check_launch(h, "pass2_dcgs");
          continue;
        }
        if (split) {
          launch_dots_split(c, j, 1, st);
          check_launch(h, "dots_split");
          launch_reduce_dots_split(c, j, 1, st);
          check_launch(h, "reduce_dots_split");
          tm.mark(C_UPDATE);
          // q_{j+1} for the vectors that take no second pass, w' for the rest
          launch_update_split(c, j, 1, st);
          check_launch(h, "update_split");
          tm.mark(C_PASS2);
          launch_dots_split(c, j, 2, st);
          check_launch(h, "dots_split2");
          launch_reduce_dots_split(c, j, 2, st);
          check_launch(h, "reduce_dots_split2");
          launch_update_split(c, j, 2, st);
          check_launch(h, "update_split2");
          continue;
        }
        launch_alpha_reduce(c, j, st);
        check_launch(h, "alpha_reduce");
        launch_alpha_axpy(c, j, st);
        check_launch(h, "alpha_axpy");
        if (reorth) {
          launch_reduce_dots(c, j, 1, st);
          check_launch(h, "reduce_dots");
          tm.mark(C_UPDATE);
          launch_update(c, j, 1, st);
          check_launch(h, "update");
          tm.mark(C_PASS2);
          launch_second_pass_decide_j(c, j, st);
          check_launch(h, "second_pass_decide");
          launch_dots(c, j, 2, st);
          check_launch(h, "dots2");
          launch_reduce_dots(c, j, 2, st);
          check_launch(h, "reduce_dots2");
          launch_update(c, j, 2, st);
          check_launch(h, "update2");
        }
        tm.mark(C_NORM);
        launch_beta_vec(c, j, st);
        check_launch(h, "beta_vec");
        launch_normalize(c, j, 0, nullptr, st);
        check_launch(h, "normalize");
        if (after_step) (*after_step)(c, j);
      }
    };
    if (graph_mode) {
      char key[512];
      snprintf(key, sizeof key,
               "%s s%p B%d n%d v%d k%d p%d r%d sp%d s32%d t%.17g M%p V%p a%p b%p b0%p ke%p g%llu",
               h->ws_prefix.c_str(), (const void *)s.L64, Bs, nvec, vec0, k, o.precision,
               o.reorth, (int)split, o.split32, o.tol, (const void *)pv.d_M,
               (const void *)pv.d_V, (void *)alpha, (void *)beta, (void *)beta0, (void *)k_eff,
               h->ws_gen);
      run_graphed(h, key, sub_body);
    } else {
      sub_body();
    }
    if (after_sub) (*after_sub)(c);
  }
  tm.stop();
  if (rep) {
    tm.collect(tacc, C_N);
    int n2 = 0;
    LGW_TRY_CUDA(h, cudaMemcpy(&n2, c.n_second, sizeof(int), cudaMemcpyDeviceToHost));
    rep->n_second_pass = n2;
    rep->n_sub_batches = nsub;
    rep->b_sub = Bs;
    rep->gemm1_splits = tc ? splits_tc : splits64;
  }
}

// Interval [x_lo, x_hi] around the spectrum of C for the polynomial form:
// x_lo = min Delta^2 (a bound: C = Delta^2 + a positive semidefinite term);
// x_hi = the largest Ritz value of k_est Lanczos steps (BF16 tensor-core
// contractions when the system has them, else FP64; CGS2) from a hash start
// vector, plus the last beta, the residual norm of that step.  Synchronous.
void estimate_interval(lgw_handle *h, const SysDev &s, int k_est, double &lo, double &hi) {
  cudaStream_t &st = h->stream;
  Opts o{};
  o.k = std::max(1, std::min(k_est, s.n_vc));
  o.precision = (s.Lb && tc_available()) ? LGW_BF16 : LGW_FP64;
  o.reorth = LGW_REORTH_CGS2;
  o.b_sub = 1;
  o.qp_max_iter = 50;
  o.split = o.precision != LGW_FP64;
  o.tol = 1e-13;
  o.qp_tol = 1e-10;
  const bool timing = h->timing;
  h->timing = false;
  double *vec = wsT<double>(h, "iv_vec", (size_t)s.n_vc);
  launch_interval(nullptr, s.n_vc, s.n_vc, nullptr, nullptr, nullptr, nullptr, vec,
                  0x5EEDull, true, st);
  check_launch(h, "hash_vector");
  ProbView pv{};
  pv.n_t = 1;
  pv.n_m = 1;
  pv.B = 1;
  pv.d_V = vec;
  pv.delta = 1.0;
  double *a = wsT<double>(h, "iv_alpha", (size_t)o.k);
  double *b = wsT<double>(h, "iv_beta", (size_t)o.k);
  double *b0 = wsT<double>(h, "iv_beta0", 1);
  int *ke = wsT<int>(h, "iv_keff", 1);
  run_lanczos(h, s, pv, o, a, b, b0, ke, nullptr, nullptr);
  double *out = wsT<double>(h, "iv_out", 2);
  launch_interval(s.Delta2, s.n_vc, s.N, a, b, ke, out, nullptr, 0, false, st);
  check_launch(h, "interval");
  double hv[2];
  LGW_TRY_CUDA(h, cudaMemcpyAsync(hv, out, sizeof hv, cudaMemcpyDeviceToHost, st));
  LGW_TRY_CUDA(h, cudaStreamSynchronize(st));
  h->timing = timing;
  lo = hv[0];
  hi = hv[1];
  if (!(lo > 0.0) || !(hi > lo)) {
    set_err(h, LGW_ERR_NOT_SPD, "spectral interval estimate [%g, %g] is not positive", lo, hi);
    throw Fail{LGW_ERR_NOT_SPD};
  }
}

// Band Lanczos over the request's targets (band width p = n_t): one
// recurrence per summed orbital g, started from [b_{t,g} over t].  Outputs
// the banded T, R0 and the step counts: Tb [G][k][p+1], R0 [G][p][p],
// keff [G] (device).  FP64 basis, CGS2; FP64 or BF16 contractions.
void run_band(lgw_handle *h, const SysDev &s, const ProbView &pv, const Opts &o, double *Tb,
              double *R0, int *keff, double *tacc) {
  cudaStream_t &st = h->stream;
  const int p = pv.n_t, G = pv.n_m, k = o.k;
  const bool tc = o.precision != LGW_FP64;
  int nsub_req = o.b_sub > 0 ? std::min(o.b_sub, G) : std::min(G, 512);
  int Bs = round_up(nsub_req, PAD_VEC);
  if (tc) Bs = std::max(Bs, 64);
  const int N = s.N;
  const int nchunks = (N + VEC_CHUNK - 1) / VEC_CHUNK;
  const int kmax1 = k + 1;
  LGW_TRY_CUDA(h, cudaMemsetAsync(Tb, 0, sizeof(double) * (size_t)G * k * (p + 1), st));
  LGW_TRY_CUDA(h, cudaMemsetAsync(R0, 0, sizeof(double) * (size_t)G * p * p, st));
  LGW_TRY_CUDA(h, cudaMemsetAsync(keff, 0, sizeof(int) * (size_t)G, st));
  BandCtx bc{};
  VecCtx &c = bc.c;
  c.N = N;
  c.Bs = Bs;
  c.nchunks = nchunks;
  c.k = k;
  c.kmax1 = kmax1;
  c.reorth = LGW_REORTH_CGS2;
  c.ring = 0;
  c.nslots = k;
  c.tol = o.tol;
  c.Delta2 = s.Delta2;
  c.dsq = s.dsq;
  c.cd = s.cd;
  c.dsqf = s.dsqf;
  c.d2f = s.d2f;
  c.kf = s.kf;
  c.w = wsT<double>(h, "w", (size_t)Bs * N);
  c.basis = wsT<double>(h, "basis", (size_t)k * Bs * N);
  c.xh = tc ? wsT<__nv_bfloat16>(h, "xh", (size_t)Bs * N) : nullptr;
  c.dot_part = wsT<double>(h, "dot_part", (size_t)Bs * nchunks * kmax1);
  c.h = wsT<double>(h, "hcoef", (size_t)Bs * kmax1);
  c.norm_a = wsT<double>(h, "norm_a", (size_t)Bs * nchunks);
  c.norm_b = wsT<double>(h, "norm_b", (size_t)Bs * nchunks);
  c.norm_c = wsT<double>(h, "norm_c", (size_t)Bs * nchunks);
  c.status = h->d_status;
  bc.p = p;
  bc.G = G;
  bc.nv = wsT<int>(h, "band_nv", (size_t)Bs);
  bc.act = wsT<int>(h, "band_act", (size_t)Bs);
  bc.newrow = wsT<int>(h, "band_newrow", (size_t)Bs);
  bc.inv = wsT<double>(h, "band_inv", (size_t)Bs);
  bc.scale = wsT<double>(h, "band_scale", (size_t)Bs);
  bc.tmax = wsT<double>(h, "band_tmax", (size_t)Bs);
  bc.hsum = wsT<double>(h, "band_hsum", (size_t)Bs * kmax1);
  bc.Tb = Tb;
  bc.R0 = R0;
  bc.keff = keff;
  bc.xq = tc ? nullptr : wsT<double>(h, "band_xq", (size_t)Bs * N);

  double *Y64 = wsT<double>(h, "y64", (size_t)Bs * s.A);
  const int splits64 = gemm1_f64_splits(s, Bs);
  double *Yp64 = tc ? nullptr : wsT<double>(h, "yp64", (size_t)splits64 * Bs * s.A);
  float *ucd_buf = tc ? wsT<float>(h, "ucd", (size_t)Bs * N) : nullptr;
  TcPlan *plan = nullptr;
  float *Yp32 = nullptr;
  __nv_bfloat16 *Yh = nullptr;
  int splits_tc = 1;
  if (tc) {
    Yp32 = wsT<float>(h, "yp32", (size_t)64 * Bs * s.A);
    Yh = wsT<__nv_bfloat16>(h, "yh", (size_t)Bs * s.A);
    char err[256];
    plan = tc_plan_create(s, Bs, c.xh, Yp32, Yh, &splits_tc, err, sizeof err);
    if (!plan) {
      set_err(h, LGW_ERR_CUDA, "%s", err);
      throw Fail{LGW_ERR_CUDA};
    }
    if (!tc_plan_has_bf16(plan)) {
      tc_plan_destroy(plan);
      set_err(h, LGW_ERR_UNSUPPORTED, "BF16 contractions need the BF16 copies of L");
      throw Fail{LGW_ERR_UNSUPPORTED};
    }
    if (!tc_plan_autotune(plan, ucd_buf, h->d_status, st, &splits_tc)) {
      tc_plan_destroy(plan);
      set_err(h, LGW_ERR_CUDA, "tensor-core tile autotuning failed");
      throw Fail{LGW_ERR_CUDA};
    }
  }
  struct PlanGuard {
    TcPlan *p;
    ~PlanGuard() {
      if (p) tc_plan_destroy(p);
    }
  } guard{plan};
  Timer tm(h);
  for (int vec0 = 0; vec0 < G; vec0 += nsub_req) {
    const int nvec = std::min(nsub_req, G - vec0);
    c.vec0 = vec0;
    c.nvec = nvec;
    launch_band_init(bc, st);
    check_launch(h, "band_init");
    // ---- the start block, one target's vectors at a time (text after Eq. 8) ----
    for (int a = 0; a < p; ++a) {
      tm.mark(C_START);
      const size_t row0 = (size_t)a * G + vec0;
      if (pv.d_M && tc) {
        if (!launch_coupling_tc(plan, s, pv.d_M + row0 * s.n_aux, nvec, ucd_buf, h->d_status, st)) {
          set_err(h, LGW_ERR_UNSUPPORTED, "tensor-core plan without the BF16 copies of L");
          throw Fail{LGW_ERR_UNSUPPORTED};
        }
        check_launch(h, "coupling_tc");
        launch_start_from_vf(c, ucd_buf, st);
        check_launch(h, "start_from_vf");
      } else if (pv.d_M) {
        if (!s.L64) {
          set_err(h, LGW_ERR_UNSUPPORTED, "start vectors from M need the BF16 or FP64 copy of L");
          throw Fail{LGW_ERR_UNSUPPORTED};
        }
        LGW_TRY_CUDA(h, cudaMemsetAsync(Y64, 0, sizeof(double) * Bs * s.A, st));
        LGW_TRY_CUDA(h, cudaMemcpy2DAsync(Y64, sizeof(double) * s.A, pv.d_M + row0 * s.n_aux,
                                          sizeof(double) * s.n_aux, sizeof(double) * s.n_aux,
                                          nvec, cudaMemcpyDeviceToDevice, st));
        launch_gemm2_f64(s, Y64, Bs, EPI_START, nullptr, nullptr, nullptr, c.w, nullptr, st);
        check_launch(h, "gemm2_f64(start)");
      } else {
        launch_start_from_v(c, pv.d_V + row0 * s.n_vc, s.n_vc, s.n_vc, st);
        check_launch(h, "start_from_v");
      }
      tm.mark(C_DOTS);
      launch_band_activate(bc, 0, a, st);
      h->launches += launch_band_append(bc, 0, a, st);
      check_launch(h, "band_append(start)");
    }
    // ---- k steps: C q_j, projected out of all of the group's vectors ----
    for (int j = 0; j < k; ++j) {
      tm.mark(C_GEMM1);
      launch_band_activate(bc, 1, j, st);
      launch_band_operand(bc, j, st);
      check_launch(h, "band_operand");
      if (tc) {
        launch_gemm1_tc(plan, h->d_status, st);
        check_launch(h, "gemm1_tc");
        launch_reduce_y_bf16(Yp32, splits_tc, Bs, s.A, Yh, nullptr, st);
        check_launch(h, "reduce_y");
        tm.mark(C_GEMM2);
        launch_gemm2_tc_split(plan, ucd_buf, h->d_status, st);
        check_launch(h, "gemm2_tc");
        launch_band_assemble(bc, j, ucd_buf, st);
        check_launch(h, "band_assemble");
      } else {
        launch_gemm1_f64(s, bc.xq, Bs, Yp64, splits64, st);
        check_launch(h, "gemm1_f64");
        launch_reduce_y_f64(Yp64, splits64, Bs, s.A, Y64, st);
        check_launch(h, "reduce_y_f64");
        tm.mark(C_GEMM2);
        launch_gemm2_f64(s, Y64, Bs, EPI_APPLY, bc.xq, nullptr, nullptr, c.w, nullptr, st);
        check_launch(h, "gemm2_f64");
      }
      tm.mark(C_DOTS);
      h->launches += launch_band_append(bc, 1, j, st);
      check_launch(h, "band_append");
    }
    launch_band_finish(bc, st);
    check_launch(h, "band_finish");
  }
  tm.stop();
  if (tacc) tm.collect(tacc, C_N);
}

void run_sigma(lgw_handle *h, const SysDev &s, const ProbView &pv, const Opts &o,
               const double *alpha, const double *beta, const double *beta0, const int *k_eff,
               double *sigma, double *e_qp, double *z_qp, lgw_report *rep, double *tacc,
               int cfmode = 0) {
  // cfmode 0: spectral map of C's tridiagonals (Omega-space fractions);
  // 1: D = p_g(C)'s own tridiagonal, (G(zeta) - G(0)) / z; 2: A's own
  // tridiagonal (Tamm-Dancoff), -eta G(zeta)
  const bool poly = cfmode != 0;
  cudaStream_t st = h->stream;
  const int B = pv.B, k = o.k;
  Timer tm(h);
  JacobiBufs jb;
  jb.a = wsT<double>(h, "jac_a", (size_t)std::max(B, 1) * k);
  jb.b2 = wsT<double>(h, "jac_b2", (size_t)std::max(B, 1) * k);
  jb.w0 = wsT<double>(h, "jac_w0", (size_t)std::max(B, 1));
  jb.n = wsT<int>(h, "jac_n", (size_t)std::max(B, 1));
  double *scratch = wsT<double>(h, "spec_scratch", (size_t)3 * std::max(B, 1) * k);
  unsigned long long *mt = wsT<unsigned long long>(h, "min_theta", 1);
  const double big = 1e300;
  unsigned long long bigbits;
  std::memcpy(&bigbits, &big, sizeof big);
  LGW_TRY_CUDA(h, cudaMemcpyAsync(mt, &bigbits, sizeof bigbits, cudaMemcpyHostToDevice, st));
  tm.mark(C_SPEC);
  if (B > 0 && poly) {
    // the fractions run on D = p_g(C)'s own tridiagonal (no spectral map)
    jb.a = const_cast<double *>(alpha);
    jb.g0 = cfmode == 1 ? wsT<double>(h, "jac_g0", (size_t)B) : nullptr;
    launch_poly_prep(alpha, beta, beta0, k_eff, B, k, jb, h->d_status, st);
    check_launch(h, "poly_prep");
  } else if (B > 0) {
    launch_spectral_impl(alpha, beta, beta0, k_eff, B, k, jb, scratch, mt, h->d_status, st);
    check_launch(h, "spectral");
  }
  CfProblem cp{};
  cp.n_t = pv.n_t;
  cp.n_m = pv.n_m;
  cp.n_freq = pv.n_freq;
  cp.k = k;
  cp.targets = pv.d_targets;
  cp.m_idx = pv.d_m_idx;
  cp.eps = s.eps;
  cp.n_v = s.n_v;
  cp.omega = pv.d_omega;
  cp.delta = pv.delta;
  cp.shift = pv.d_shift;
  cp.qp_mode = o.qp_mode;
  tm.mark(C_CF);
  double *sig = sigma ? sigma : wsT<double>(h, "sigma_tmp", (size_t)std::max(1, pv.n_t * pv.n_freq * 2));
  const int S = cf_slices(cp);
  double *part = S > 1 ? wsT<double>(h, "cf_part", (size_t)S * pv.n_t * pv.n_freq * 2) : nullptr;
  const int ncf = launch_cf_grid(cp, jb, sig, part, S, st);
  if (ncf > 0) check_launch(h, "cf_grid");
  if (ncf > 1) check_launch(h, "cf_reduce");
  tm.mark(C_QP);
  if (e_qp && pv.n_t > 0) {
    launch_qp(cp, jb, sig, o.qp_max_iter, o.qp_tol, e_qp, z_qp, h->d_status, st);
    check_launch(h, "qp");
  }
  tm.stop();
  if (rep) {
    tm.collect(tacc, C_N);
    unsigned long long bits = 0;
    LGW_TRY_CUDA(h, cudaMemcpy(&bits, mt, sizeof bits, cudaMemcpyDeviceToHost));
    double mtv;
    std::memcpy(&mtv, &bits, sizeof mtv);
    rep->min_theta = mtv;
  }
}

void fill_report_common(lgw_handle *h, const SysDev &s, const ProbView &pv, const Opts &o,
                        const int *k_eff_dev, lgw_report *rep, const double *tacc) {
  if (!rep) return;
  rep->ms_start = tacc[C_START];
  rep->ms_gemm1 = tacc[C_GEMM1];
  rep->ms_gemm2 = tacc[C_GEMM2];
  rep->ms_dots = tacc[C_DOTS];
  rep->ms_update = tacc[C_UPDATE];
  rep->ms_pass2 = tacc[C_PASS2];
  rep->ms_normalize = tacc[C_NORM];
  rep->ms_spectral = tacc[C_SPEC];
  rep->ms_cf = tacc[C_CF];
  rep->ms_qp = tacc[C_QP];
  rep->n_vectors = pv.B;
  std::vector<int> ke(pv.B);
  if (pv.B) {
    LGW_TRY_CUDA(h, cudaMemcpy(ke.data(), k_eff_dev, sizeof(int) * pv.B, cudaMemcpyDeviceToHost));
  }
  int kmin = o.k, kmax = 0;
  double elems = 0.0;
  for (int x : ke) {
    kmin = std::min(kmin, x);
    kmax = std::max(kmax, x);
    elems += (double)s.n_vc * (double)x * (double)(x + 1) / 2.0;
  }
  rep->k_min = pv.B ? kmin : 0;
  rep->k_max = kmax;
  rep->gemm_flops = 4.0 * s.n_vc * (double)s.n_aux * (double)pv.B * (double)o.k;
  rep->reorth_elems = o.reorth != LGW_REORTH_NONE ? elems : 0.0;
}

lgw_status guard_handle(lgw_handle *h) {
  if (!h) return LGW_ERR_ARG;
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return set_err(h, LGW_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  h->last = LGW_OK;
  h->msg.clear();
  return LGW_OK;
}

}  // namespace

// ===========================================================================
// exported C ABI
// ===========================================================================
namespace {
// x_lo = x_hi = 0 asks the library for the interval (estimate_interval,
// kept with the system after its first estimate).
const PolyOp *poly_arg(lgw_handle *h, const lgw_system *sys, const lgw_poly *pp, PolyOp &store) {
  if (!pp) return nullptr;
  double lo = pp->x_lo, hi = pp->x_hi;
  if (pp->g >= 1 && pp->g <= 256 && lo == 0.0 && hi == 0.0) {
    lgw_system *ms = const_cast<lgw_system *>(sys);
    if (!ms->ivl_ok) {
      estimate_interval(h, sys->s, 32, ms->ivl_lo, ms->ivl_hi);
      ms->ivl_ok = true;
    }
    lo = ms->ivl_lo;
    hi = ms->ivl_hi;
  }
  if (pp->g < 1 || pp->g > 256 || !(lo > 0.0) || !(hi > lo)) {
    set_err(h, LGW_ERR_ARG, "polynomial: need 1 <= g <= 256 and 0 < x_lo < x_hi (or both 0)");
    throw Fail{LGW_ERR_ARG};
  }
  store = make_poly(pp->g, lo, hi);
  return &store;
}

// Tamm-Dancoff view of a system: the same copies of L with Delta^1/2 -> 1,
// Delta^2 -> Delta, c_K Delta^1/2 -> c_K / 2 (refreshed on every use, so
// copies made later, such as the E4M3 ones, are seen).
const SysDev &tda_view(lgw_handle *h, const lgw_system *csys) {
  lgw_system *sys = const_cast<lgw_system *>(csys);
  const SysDev &s = sys->s;
  if (!sys->tda_buf) {
    const size_t N = (size_t)s.N;
    void *buf = nullptr;
    LGW_TRY_CUDA(h, cudaMalloc(&buf, N * (2 * sizeof(double) + 4 * sizeof(float))));
    sys->tda_buf = buf;
    double *ones = static_cast<double *>(buf), *cd = ones + N;
    float *onesf = reinterpret_cast<float *>(cd + N), *d2f = onesf + N, *cdf = d2f + N;
    launch_tda_view(s.Delta, s.n_vc, s.N, 0.5 * s.kf, ones, cd, onesf, d2f, cdf + N, cdf,
                    h->stream);
    check_launch(h, "tda_view");
  }
  const size_t N = (size_t)s.N;
  double *ones = static_cast<double *>(sys->tda_buf), *cd = ones + N;
  float *onesf = reinterpret_cast<float *>(cd + N), *d2f = onesf + N, *cdf = d2f + N;
  SysDev &t = sys->tda;
  t = s;
  t.kf = 0.5 * s.kf;
  t.dsq = ones;
  t.Delta2 = s.Delta;
  t.cd = cd;
  t.dsqf = onesf;
  t.d2f = d2f;
  t.d2lo = cdf + N;
  t.cdf = cdf;
  return t;
}

lgw_status sigma_c_impl(lgw_handle *h, const lgw_system *sys, const lgw_problem *p,
                        const lgw_options *o, const lgw_poly *pp, double *sigma, double *e_qp,
                        double *z_qp, lgw_report *rep, bool tda = false) {
  lgw_status g = guard_handle(h);
  if (g != LGW_OK) return g;
  if (!sys || sys->h != h) return set_err(h, LGW_ERR_ARG, "bad system handle");
  try {
    cudaStream_t st = h->stream;
    h->launches = 0;
    h->ev_used = 0;
    h->timing = rep != nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (rep) {
      std::memset(rep, 0, sizeof *rep);
      LGW_TRY_CUDA(h, cudaEventCreate(&t0));
      LGW_TRY_CUDA(h, cudaEventCreate(&t1));
      LGW_TRY_CUDA(h, cudaEventRecord(t0, st));
    }
    LGW_TRY_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), st));
    Opts op = resolve_opts(h, o, sys->s);
    ensure_copies(h, sys, op);
    PolyOp pstore;
    const PolyOp *poly = poly_arg(h, sys, pp, pstore);
    if (poly) {
      // Lanczos on D = p_g(C) keeps the FP64 basis
      op.split = 0;
      op.split32 = 0;
    }
    const SysDev &s = tda ? tda_view(h, sys) : sys->s;
    ProbView pv = check_problem(h, s, p);
    double tacc[C_N] = {0};
    double *alpha = wsT<double>(h, "co_alpha", (size_t)std::max(1, pv.B) * op.k);
    double *beta = wsT<double>(h, "co_beta", (size_t)std::max(1, pv.B) * op.k);
    double *beta0 = wsT<double>(h, "co_beta0", (size_t)std::max(1, pv.B));
    int *ke = wsT<int>(h, "co_keff", (size_t)std::max(1, pv.B));
    OutBuf<double> sg, e, z;
    sg.init(h, "out_sigma", sigma, (size_t)pv.n_t * pv.n_freq * 2);
    e.init(h, "out_eqp", e_qp, (size_t)pv.n_t);
    z.init(h, "out_zqp", z_qp, (size_t)pv.n_t);
    run_lanczos(h, s, pv, op, alpha, beta, beta0, ke, rep, tacc, false, nullptr, poly);
    run_sigma(h, s, pv, op, alpha, beta, beta0, ke, sg.dev, e.dev, z.dev, rep, tacc,
              poly != nullptr ? 1 : (tda ? 2 : 0));
    sg.finish(h);
    e.finish(h);
    z.finish(h);
    if (rep) {
      LGW_TRY_CUDA(h, cudaEventRecord(t1, st));
      LGW_TRY_CUDA(h, cudaEventSynchronize(t1));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, t0, t1);
      cudaEventDestroy(t0);
      cudaEventDestroy(t1);
      fill_report_common(h, s, pv, op, ke, rep, tacc);
      if (poly) rep->gemm_flops *= poly->g;
      rep->ms_total = ms;
      rep->gpu_launches = h->launches;
    }
    check_status(h);
    h->timing = false;
  } catch (Fail &f) {
    h->timing = false;
    return f.st;
  }
  return LGW_OK;
}
// Exact reverse mode of one sub-batch's three-term recurrence (FP64, no
// reorthogonalisation), segment by segment from the last: each segment
// [s0, s0 + ci) is recomputed from its checkpoint (q_{s0-1}, q_s0) with the
// forward's own kernels (breakdown test off: the recorded depths stand),
// then taken back step by step (k_rev_*: one dot pass, one scalar step, one
// elementwise pass, and C ubar_j through the FP64 contractions).  SC
// accumulates sum_j (ubar_j (L^T D q_j)^T + q_j (L^T D ubar_j)^T) = 2 G D L;
// then y = dF/db, SB += y M^T and the diagonal terms of dDelta.
//
// Polynomial form (poly != NULL: the recurrence runs on D = p_g(C)): each
// product D x is Clenshaw's recurrence in S = a_s C + b_s I (g products with
// C).  Taking step j back needs D ubar_j and the pairs through which dF/dD
// reaches C: Clenshaw on q_j is redone (b_1..b_g and their L^T D b_k), then
// the reverse recurrence bbar_1 = S u, bbar_k = 2 S bbar_{k-1} - bbar_{k-2}
// (u = bbar_0 = ubar_j) gives D u = c_0 u + sum_k c_k bbar_k and
//   dF/dC += a_s u b_1^T + 2 a_s sum_{k=1}^{g-1} bbar_k b_{k+1}^T.
void reverse_sweep(lgw_handle *h, const SysDev &s, const ProbView &pv, const Opts &op,
                   const VecCtx &c, const AdjCtx &a, const double *ckpt, int ci, double *SC,
                   double *SB, double *dD, double *gdeps, const PolyOp *poly) {
  cudaStream_t &st = h->stream;
  const int Bs = c.Bs, N = c.N, A = s.A, k = op.k;
  const size_t BN = (size_t)Bs * N, BA = (size_t)Bs * A;
  const int cs = std::min(ci, k), nseg = (k + ci - 1) / ci;
  double *seg = wsT<double>(h, "rev_seg", (size_t)(cs + 2) * BN);
  double *useg = wsT<double>(h, "rev_useg", (size_t)cs * BN);
  double *yseg = wsT<double>(h, "rev_yseg", (size_t)cs * BA);
  double *ybseg = wsT<double>(h, "rev_ybseg", (size_t)cs * BA);
  const int sp = gemm1_f64_splits(s, Bs);
  double *yp = wsT<double>(h, "rev_yp", (size_t)sp * BA);
  double *Y = wsT<double>(h, "adj_Y", BN);
  RevCtx r{};
  r.N = N;
  r.Bs = Bs;
  r.nvec = c.nvec;
  r.vec0 = c.vec0;
  r.k = k;
  r.nchunks = c.nchunks;
  r.seg = seg;
  r.qbar = wsT<double>(h, "rev_qbar", 3 * BN);
  double *cu = wsT<double>(h, "rev_cu", BN);
  r.cu = cu;
  r.useg = useg;
  r.Gd = wsT<double>(h, "adj_Gd", BN);
  // on D = p_g(C) the pairs of the reverse Clenshaw recurrence give diag(dF/dC)
  r.gd_from_steps = poly ? 0 : 1;
  r.dpart = wsT<double>(h, "rev_dpart", (size_t)Bs * c.nchunks * 6);
  r.coef = wsT<double>(h, "rev_coef", (size_t)Bs * 8);
  r.bbar = wsT<double>(h, "rev_bbar", (size_t)Bs * k);
  r.Gam = a.Gam;
  r.ay = a.ay;
  r.alpha = a.alpha;
  r.beta = a.beta;
  r.beta0 = a.beta0;
  r.k_eff = a.k_eff;
  LGW_TRY_CUDA(h, cudaMemsetAsync(r.qbar, 0, sizeof(double) * 3 * BN, st));
  LGW_TRY_CUDA(h, cudaMemsetAsync(cu, 0, sizeof(double) * BN, st));
  LGW_TRY_CUDA(h, cudaMemsetAsync(r.Gd, 0, sizeof(double) * BN, st));
  launch_rev_init(r, st);
  check_launch(h, "rev_init");
  // polynomial form: Clenshaw vectors b_k (slot k - 1), their L^T D b_k, the
  // reverse vectors bbar_1..bbar_g (slot k - 1) and L^T D bbar_{k-1}
  const int g = poly ? poly->g : 0;
  double *fb = nullptr, *fy = nullptr, *rb = nullptr, *ry = nullptr, *T = nullptr,
         *apart = nullptr, *zeros = nullptr;
  if (poly) {
    fb = wsT<double>(h, "rev_fb", (size_t)g * BN);
    fy = wsT<double>(h, "rev_fy", (size_t)g * BA);
    rb = wsT<double>(h, "rev_rb", (size_t)g * BN);
    ry = wsT<double>(h, "rev_ry", (size_t)g * BA);
    T = wsT<double>(h, "rev_T", BN);
    apart = wsT<double>(h, "rev_apart", (size_t)c.nchunks * Bs);
    zeros = wsT<double>(h, "rev_zeros", (size_t)Bs);
    LGW_TRY_CUDA(h, cudaMemsetAsync(zeros, 0, sizeof(double) * Bs, st));
  }
  // T = C x with L^T D x into yout (FP64 contractions)
  auto apply_c = [&](const double *x, double *yout) {
    launch_gemm1_f64(s, x, Bs, yp, sp, st);
    check_launch(h, "gemm1_f64(reverse)");
    launch_reduce_y_f64(yp, sp, Bs, A, yout, st);
    check_launch(h, "reduce_y_f64(reverse)");
    launch_gemm2_f64(s, yout, Bs, EPI_APPLY, x, nullptr, nullptr, T, nullptr, st);
    check_launch(h, "gemm2_f64(reverse)");
  };
  auto fbk = [&](int k) { return fb + (size_t)(k - 1) * BN; };
  auto rbk = [&](int k) { return rb + (size_t)(k - 1) * BN; };
  // Clenshaw on x: b_g .. b_1 into fb and L^T D b_k into fy; with w given,
  // also the Lanczos step's w = D x - beta_j q_{j-1} and its alpha partials
  auto clenshaw = [&](const double *x, const double *qprev, const double *betaj, double *w,
                      double *alpha_part) {
    PolyStep ps{};
    ps.N = N;
    ps.q = x;
    ps.Delta2 = s.Delta2;
    ps.dsqf = s.dsqf;
    ps.as = poly->as;
    ps.bs = poly->bs;
    ps.ck = poly->c[g];
    ps.out = fbk(g);
    launch_cheb_step(ps, c.nchunks, Bs, st);
    check_launch(h, "cheb_step(reverse)");
    for (int kk = g - 1; kk >= 0; --kk) {
      apply_c(fbk(kk + 1), fy + (size_t)kk * BA);
      ps.b1 = fbk(kk + 1);
      ps.b2 = kk + 2 <= g ? fbk(kk + 2) : nullptr;
      ps.T = T;
      ps.ck = poly->c[kk];
      if (kk > 0) {
        ps.out = fbk(kk);
        launch_cheb_step(ps, c.nchunks, Bs, st);
        check_launch(h, "cheb_step(reverse)");
      } else if (w) {
        ps.out = nullptr;
        launch_cheb_final(ps, qprev, betaj, w, alpha_part, c.nchunks, Bs, st);
        check_launch(h, "cheb_final(reverse)");
      }
    }
  };
  // the recomputation window: q_j at slot j - (s0 - 1) of seg
  VecCtx rc = c;
  rc.ring = 0;
  rc.basis = seg;
  rc.nslots = cs + 2;
  rc.tol = 0.0;
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int s0 = sg * ci, e = std::min(s0 + ci, k), n = e - s0;
    LGW_TRY_CUDA(h, cudaMemcpyAsync(seg, ckpt + (size_t)sg * 2 * BN, sizeof(double) * 2 * BN,
                                    cudaMemcpyDeviceToDevice, st));
    rc.slot0 = s0 - 1;
    r.s0 = s0;
    launch_rev_set_betaj(r, rc.betaj, st);
    check_launch(h, "rev_set_betaj");
    for (int j = s0; j < e; ++j) {
      const double *qj = slot_ptr(rc, j);
      const double *qp = j > 0 ? slot_ptr(rc, j - 1) : nullptr;
      if (poly) {
        clenshaw(qj, qp, rc.betaj, rc.w, rc.alpha_part);
      } else {
        double *yj = yseg + (size_t)(j - s0) * BA;
        launch_gemm1_f64(s, qj, Bs, yp, sp, st);
        check_launch(h, "gemm1_f64(recompute)");
        launch_reduce_y_f64(yp, sp, Bs, A, yj, st);
        check_launch(h, "reduce_y_f64(recompute)");
        launch_gemm2_f64(s, yj, Bs, EPI_LANCZOS, qj, qp, rc.betaj, rc.w, rc.alpha_part, st);
        check_launch(h, "gemm2_f64(recompute)");
      }
      launch_alpha_reduce(rc, j, st);
      check_launch(h, "alpha_reduce(recompute)");
      launch_alpha_axpy(rc, j, st);
      check_launch(h, "alpha_axpy(recompute)");
      launch_beta_vec(rc, j, st);
      check_launch(h, "beta_vec(recompute)");
      launch_normalize(rc, j, 0, nullptr, st);
      check_launch(h, "normalize(recompute)");
    }
    for (int j = e - 1; j >= s0; --j) {
      launch_rev_step(r, j, st);
      check_launch(h, "rev_step");
      const double *uj = useg + (size_t)(j - s0) * BN;
      if (!poly) {
        double *ybj = ybseg + (size_t)(j - s0) * BA;
        launch_gemm1_f64(s, uj, Bs, yp, sp, st);
        check_launch(h, "gemm1_f64(reverse)");
        launch_reduce_y_f64(yp, sp, Bs, A, ybj, st);
        check_launch(h, "reduce_y_f64(reverse)");
        launch_gemm2_f64(s, ybj, Bs, EPI_APPLY, uj, nullptr, nullptr, cu, nullptr, st);
        check_launch(h, "gemm2_f64(reverse)");
        continue;
      }
      // Clenshaw vectors of q_j, then the reverse recurrence from u = ubar_j
      clenshaw(slot_ptr(rc, j), nullptr, nullptr, nullptr, nullptr);
      PolyStep ps{};
      ps.N = N;
      ps.q = uj;
      ps.Delta2 = s.Delta2;
      ps.dsqf = s.dsqf;
      ps.as = poly->as;
      ps.bs = poly->bs;
      ps.ck = 0.0;
      apply_c(uj, ry);
      ps.b1 = uj;
      ps.T = T;
      launch_cheb_final(ps, nullptr, zeros, rbk(1), apart, c.nchunks, Bs, st);   // S u
      check_launch(h, "cheb_final(reverse S u)");
      for (int kk = 2; kk <= g; ++kk) {
        apply_c(rbk(kk - 1), ry + (size_t)(kk - 1) * BA);
        ps.b1 = rbk(kk - 1);
        ps.b2 = kk == 2 ? uj : rbk(kk - 2);
        ps.out = rbk(kk);
        launch_cheb_step(ps, c.nchunks, Bs, st);
        check_launch(h, "cheb_step(reverse)");
      }
      // D u for qbar_j (added by the next step's first pass)
      launch_rev_axpby(cu, poly->c[0], uj, 0.0, BN, st);
      for (int kk = 1; kk <= g; ++kk) launch_rev_axpby(cu, poly->c[kk], rbk(kk), 1.0, BN, st);
      check_launch(h, "rev_axpby");
      // pairs (a_s: u, b_1) and (2 a_s: bbar_k, b_{k+1}), k = 1 .. g-1
      const double as = poly->as;
      launch_rev_gd(r.Gd, as, uj, fbk(1), BN, st);
      for (int kk = 1; kk < g; ++kk) launch_rev_gd(r.Gd, 2.0 * as, rbk(kk), fbk(kk + 1), BN, st);
      check_launch(h, "rev_gd");
      launch_atb_f64(uj, N, fy, A, Bs, N, A, SC, st, as);
      launch_atb_f64(fbk(1), N, ry, A, Bs, N, A, SC, st, as);
      if (g > 1) {
        launch_atb_f64(rbk(1), N, fy + BA, A, (g - 1) * Bs, N, A, SC, st, 2.0 * as);
        launch_atb_f64(fbk(2), N, ry + BA, A, (g - 1) * Bs, N, A, SC, st, 2.0 * as);
      }
      check_launch(h, "atb_f64(SC, poly pairs)");
    }
    if (poly) continue;
    launch_atb_f64(useg, N, yseg, A, n * Bs, N, A, SC, st);
    check_launch(h, "atb_f64(SC, ubar)");
    launch_atb_f64(seg + BN, N, ybseg, A, n * Bs, N, A, SC, st);
    check_launch(h, "atb_f64(SC, q)");
  }
  const double *q0 = ckpt + BN;
  launch_rev_finish(r, q0, Y, st);
  check_launch(h, "rev_finish");
  if (SB) {
    launch_atb_f64(Y, N, pv.d_M + (size_t)c.vec0 * s.n_aux, s.n_aux, c.nvec, N, s.n_aux, SB, st);
    check_launch(h, "atb_f64(SB)");
  }
  launch_adj_accumulate(a, s.Delta, BasisRef{q0, nullptr, nullptr}, Y, r.Gd, dD, gdeps, st);
  check_launch(h, "adj_accumulate");
}
}  // namespace

extern "C" {

const char *lgw_status_string(lgw_status s) {
  switch (s) {
    case LGW_OK: return "ok";
    case LGW_ERR_ARG: return "invalid argument";
    case LGW_ERR_SHAPE: return "inconsistent shape or index";
    case LGW_ERR_CUDA: return "CUDA error";
    case LGW_ERR_OOM: return "out of device memory";
    case LGW_ERR_NOT_SPD: return "Casida matrix or Gauss node not positive";
    case LGW_ERR_NO_CONVERGENCE: return "no convergence";
    case LGW_ERR_TIMEOUT: return "device wait timed out";
    case LGW_ERR_UNSUPPORTED: return "unsupported option";
  }
  return "unknown status";
}

lgw_status lgw_create(lgw_handle **out, int device, void *cuda_stream) {
  if (!out) return LGW_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return LGW_ERR_ARG;
  }
  if (cudaSetDevice(device) != cudaSuccess) return LGW_ERR_CUDA;
  lgw_handle *h = new lgw_handle();
  h->device = device;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaMalloc(&h->d_status, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return LGW_ERR_OOM;
  }
  cudaMemset(h->d_status, 0, sizeof(unsigned));
  *out = h;
  return LGW_OK;
}

lgw_status lgw_destroy(lgw_handle *h) {
  if (!h) return LGW_OK;
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  h->drop_graphs();
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (auto l : h->lanes) cudaStreamDestroy(l);
  for (auto &kv : h->bufs)
    if (kv.second.p) cudaFree(kv.second.p);
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  if (h->d_status) cudaFree(h->d_status);
  delete h;
  return LGW_OK;
}

lgw_status lgw_set_workspace_limit(lgw_handle *h, size_t bytes) {
  lgw_status g = guard_handle(h);
  if (g != LGW_OK) return g;
  h->ws_limit = bytes;
  return LGW_OK;
}

lgw_status lgw_workspace_bytes(lgw_handle *h, size_t *bytes) {
  lgw_status g = guard_handle(h);
  if (g != LGW_OK) return g;
  if (!bytes) return set_err(h, LGW_ERR_ARG, "NULL argument to lgw_workspace_bytes");
  *bytes = h->ws_bytes;
  return LGW_OK;
}

lgw_status lgw_release_workspace(lgw_handle *h) {
  lgw_status g = guard_handle(h);
  if (g != LGW_OK) return g;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess)
    return set_err(h, LGW_ERR_CUDA, "stream synchronisation before the release failed");
  h->drop_graphs();
  for (auto &kv : h->bufs)
    if (kv.second.p) cudaFree(kv.second.p);
  h->bufs.clear();
  h->ws_bytes = 0;
  h->ws_gen++;
  return LGW_OK;
}

lgw_status lgw_selftest_bounded_wait(lgw_handle *h, int32_t arrive, double seconds) {
  lgw_status g = guard_handle(h);
  if (g != LGW_OK) return g;
  if (!(seconds >= 1e-4 && seconds <= 2.0))
    return set_err(h, LGW_ERR_ARG, "self-test wait must lie in [1e-4, 2] s");
  int khz = 0;
  if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, h->device) != cudaSuccess || khz <= 0)
    return set_err(h, LGW_ERR_CUDA, "clock rate query failed");
  const long long cycles = (long long)(seconds * (double)khz * 1e3);
  cudaStream_t st = h->stream;
  if (cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), st) != cudaSuccess)
    return set_err(h, LGW_ERR_CUDA, "status reset failed");
  launch_wait_selftest(arrive != 0, cycles, h->d_status, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return set_err(h, LGW_ERR_CUDA, "self-test launch failed: %s", cudaGetErrorString(e));
  unsigned stw = 0;
  if (cudaMemcpyAsync(&stw, h->d_status, sizeof stw, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return set_err(h, LGW_ERR_CUDA, "self-test status read failed");
  if (stw & ST_TIMEOUT)
    return set_err(h, LGW_ERR_TIMEOUT, "a bounded device wait ran out (self-test, %.3g s)",
                   seconds);
  return LGW_OK;
}

lgw_status lgw_last_error(lgw_handle *h, char *buf, size_t n) {
  if (!h) return LGW_ERR_ARG;
  if (buf && n) {
    std::strncpy(buf, h->msg.c_str(), n - 1);
    buf[n - 1] = '\0';
  }
  return h->last;
}

lgw_status lgw_prepare_system(lgw_handle *h, const lgw_system_desc *d, lgw_system **out) {
  lgw_status g = guard_handle(h);
  if (g != LGW_OK) return g;
  if (!d || !out || !d->eps || !d->L) return set_err(h, LGW_ERR_ARG, "NULL descriptor field");
  if (d->n_v < 1 || d->n_c < 1 || d->n_aux < 1)
    return set_err(h, LGW_ERR_ARG, "n_v, n_c, n_aux must be >= 1");
  // the 32 x 32 transpose tiles of the operand copies use grid.y = N / 32
  if ((int64_t)d->n_v * d->n_c > (int64_t)65535 * 32)
    return set_err(h, LGW_ERR_SHAPE, "n_v * n_c above 2097120");
  if (!(d->kernel_factor >= 0.0)) return set_err(h, LGW_ERR_ARG, "kernel_factor must be >= 0");
  *out = nullptr;
  lgw_system *sys = new lgw_system();
  sys->h = h;
  SysDev &s = sys->s;
  s.n_v = d->n_v;
  s.n_c = d->n_c;
  s.n_aux = d->n_aux;
  s.n_vc = d->n_v * d->n_c;
  s.N = round_up(s.n_vc, PAD_VC);
  s.A = round_up(s.n_aux, PAD_AUX);
  s.kf = d->kernel_factor;
  std::vector<void *> allocs;
  auto alloc = [&](size_t bytes) -> void * {
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    allocs.push_back(p);
    return p;
  };
  const int flags = d->flags;
  if ((flags & ~(LGW_SYS_NO_FP64 | LGW_SYS_NO_BF16 | LGW_SYS_FP8)) != 0 ||
      ((flags & LGW_SYS_NO_FP64) && (flags & LGW_SYS_NO_BF16))) {
    delete sys;
    return set_err(h, LGW_ERR_ARG, "bad system flags 0x%x", flags);
  }
  const bool keep64 = !(flags & LGW_SYS_NO_FP64), keep16 = !(flags & LGW_SYS_NO_BF16);
  const int norb = s.n_v + s.n_c;
  s.eps = (double *)alloc(sizeof(double) * norb);
  s.Delta = (double *)alloc(sizeof(double) * s.N);
  s.dsq = (double *)alloc(sizeof(double) * s.N);
  s.Delta2 = (double *)alloc(sizeof(double) * s.N);
  s.cd = (double *)alloc(sizeof(double) * s.N);
  s.dsqf = (float *)alloc(sizeof(float) * s.N);
  s.d2f = (float *)alloc(2 * sizeof(float) * s.N);   // d2f, then d2lo
  s.d2lo = s.d2f ? s.d2f + s.N : nullptr;
  s.cdf = (float *)alloc(sizeof(float) * s.N);
  bool ok = s.eps && s.Delta && s.dsq && s.Delta2 && s.cd && s.dsqf && s.d2f && s.cdf;
  if (ok && keep64) ok = (s.L64 = (double *)alloc(sizeof(double) * (size_t)s.N * s.A)) != nullptr;
  if (ok && keep16) {
    s.Lb = (__nv_bfloat16 *)alloc(sizeof(__nv_bfloat16) * (size_t)s.N * s.A);
    s.Ltb = (__nv_bfloat16 *)alloc(sizeof(__nv_bfloat16) * (size_t)s.N * s.A);
    s.Lb_lo = (__nv_bfloat16 *)alloc(sizeof(__nv_bfloat16) * (size_t)s.N * s.A);
    ok = s.Lb && s.Ltb && s.Lb_lo;
  }
  if (!ok) {
    for (void *p : allocs) cudaFree(p);
    delete sys;
    return set_err(h, LGW_ERR_OOM, "device allocation for the system failed");
  }
  try {
    cudaStream_t st = h->stream;
    LGW_TRY_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), st));
    if (is_device_ptr(d->eps))
      LGW_TRY_CUDA(h, cudaMemcpyAsync(s.eps, d->eps, sizeof(double) * norb, cudaMemcpyDeviceToDevice, st));
    else
      LGW_TRY_CUDA(h, cudaMemcpyAsync(s.eps, d->eps, sizeof(double) * norb, cudaMemcpyHostToDevice, st));
    const double *Lsrc = in_dev(h, "in_L", d->L, (size_t)s.n_vc * s.n_aux);
    launch_pair_energies(s, st);
    check_launch(h, "pair_energies");
    launch_check_delta(s, h->d_status, st);
    check_launch(h, "check_delta");
    if (keep64) {
      launch_pad_L(Lsrc, s, st);
      check_launch(h, "pad_L");
    }
    if (keep16) {
      launch_quantize_L(Lsrc, s.n_aux, s.n_vc, s.n_aux, s, st);
      check_launch(h, "quantize_L");
    }
    if (!keep64 || (flags & LGW_SYS_FP8)) make_fp8(h, s, Lsrc, s.n_aux, s.n_vc, s.n_aux);
    check_status(h);
  } catch (Fail &f) {
    for (void *p : allocs) cudaFree(p);
    if (s.L8) cudaFree(s.L8);
    if (s.L8t) cudaFree(s.L8t);
    if (s.sL) cudaFree(s.sL);
    delete sys;
    return f.st;
  }
  *out = sys;
  return LGW_OK;
}

lgw_status lgw_release_system(lgw_system *sys) {
  if (!sys) return LGW_OK;
  cudaSetDevice(sys->h->device);
  cudaStreamSynchronize(sys->h->stream);
  // cached graphs may reference this system's buffers
  sys->h->drop_graphs();
  SysDev &s = sys->s;
  void *ps[] = {s.eps,  s.Delta, s.dsq, s.Delta2, s.cd,  s.dsqf,
                s.d2f, s.cdf,   s.L64, s.Lb,     s.Ltb, s.Lb_lo};
  for (void *p : ps)
    if (p) cudaFree(p);
  if (sys->Ltb_lo) cudaFree(sys->Ltb_lo);
  if (sys->tda_buf) cudaFree(sys->tda_buf);
  if (s.L8) cudaFree(s.L8);
  if (s.L8t) cudaFree(s.L8t);
  if (s.sL) cudaFree(s.sL);
  delete sys;
  return LGW_OK;
}

lgw_status lgw_apply_casida(lgw_handle *h, const lgw_system *sys, int32_t n_vec, const double *X,
                            double *Y, int32_t precision) {
  lgw_status g = guard_handle(h);
  if (g != LGW_OK) return g;
  if (!sys || sys->h != h || n_vec < 0 || (n_vec > 0 && (!X || !Y)))
    return set_err(h, LGW_ERR_ARG, "bad arguments to lgw_apply_casida");
  if (n_vec == 0) return LGW_OK;
  if (precision != LGW_FP64 && precision != LGW_BF16 && precision != LGW_FP8 &&
      precision != LGW_FP8_DEQ)
    return set_err(h, LGW_ERR_ARG, "bad precision");
  try {
    const SysDev &s = sys->s;
    cudaStream_t st = h->stream;
    const bool tc = precision != LGW_FP64;
    const bool fp8 = precision == LGW_FP8;
    const bool deq = precision == LGW_FP8_DEQ;
    if (tc && !tc_available()) {
      set_err(h, LGW_ERR_UNSUPPORTED, "tensor-core paths need an sm_103 device");
      throw Fail{LGW_ERR_UNSUPPORTED};
    }
    {
      Opts oa{};
      oa.precision = precision;
      ensure_copies(h, sys, oa);
    }
    LGW_TRY_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), st));
    const double *Xd = in_dev(h, "ap_xin", X, (size_t)n_vec * s.n_vc);
    OutBuf<double> Yo;
    Yo.init(h, "ap_yout", Y, (size_t)n_vec * s.n_vc);
    int Bs = round_up(n_vec, PAD_VEC);
    if (tc) Bs = std::max(Bs, 64);
    double *xp = wsT<double>(h, "ap_x", (size_t)Bs * s.N);
    double *wp = wsT<double>(h, "ap_w", (size_t)Bs * s.N);
    LGW_TRY_CUDA(h, cudaMemsetAsync(xp, 0, sizeof(double) * Bs * s.N, st));
    LGW_TRY_CUDA(h, cudaMemcpy2DAsync(xp, sizeof(double) * s.N, Xd, sizeof(double) * s.n_vc,
                                      sizeof(double) * s.n_vc, n_vec, cudaMemcpyDeviceToDevice, st));
    double *Y64 = wsT<double>(h, "y64", (size_t)Bs * s.A);
    if (tc) {
      __nv_bfloat16 *xh = wsT<__nv_bfloat16>(h, "ap_xh", (size_t)Bs * s.N);
      float *yp = wsT<float>(h, "ap_yp32", (size_t)64 * Bs * s.A);
      __nv_bfloat16 *yh = wsT<__nv_bfloat16>(h, "ap_yh", (size_t)Bs * s.A);
      launch_scale_rows_to_bf16(xp, s.dsq, Bs, s.N, xh, st);
      check_launch(h, "scale_rows_to_bf16");
      char err[256];
      int splits = 1;
      TcPlan *plan = tc_plan_create(s, Bs, xh, yp, yh, &splits, err, sizeof err);
      if (!plan) {
        set_err(h, LGW_ERR_CUDA, "%s", err);
        throw Fail{LGW_ERR_CUDA};
      }
      uint8_t *x8 = nullptr, *y8 = nullptr;
      float *sx = nullptr, *ty = nullptr;
      if (fp8) {
        x8 = wsT<uint8_t>(h, "ap_x8", (size_t)Bs * s.N);
        y8 = wsT<uint8_t>(h, "ap_y8", (size_t)Bs * s.A);
        sx = wsT<float>(h, "ap_sx", (size_t)Bs);
        ty = wsT<float>(h, "ap_ty", (size_t)Bs);
        if (!tc_plan_enable_fp8(plan, s.L8t, s.L8, x8, y8, ty)) {
          tc_plan_destroy(plan);
          set_err(h, LGW_ERR_CUDA, "cuTensorMapEncodeTiled failed for the E4M3 operands");
          throw Fail{LGW_ERR_CUDA};
        }
        launch_quant_x8(xh, Bs, s.N, x8, sx, st);
        check_launch(h, "quant_x8");
      }
      uint16_t *x16 = nullptr, *y16 = nullptr;
      if (deq) {
        x16 = wsT<uint16_t>(h, "ap_x16", (size_t)Bs * s.N);
        y16 = wsT<uint16_t>(h, "ap_y16", (size_t)Bs * s.A);
        sx = wsT<float>(h, "ap_sx", (size_t)Bs);
        ty = wsT<float>(h, "ap_ty", (size_t)Bs);
        if (!tc_plan_enable_deq(plan, s.L8t, s.L8, x16, y16, ty)) {
          tc_plan_destroy(plan);
          set_err(h, LGW_ERR_CUDA, "cuTensorMapEncodeTiled failed for the widened E4M3 operands");
          throw Fail{LGW_ERR_CUDA};
        }
        launch_quant_x16(xh, Bs, s.N, x16, sx, st);
        check_launch(h, "quant_x16");
      }
      launch_gemm1_tc(plan, h->d_status, st);
      check_launch(h, "gemm1_tc");
      if (fp8)
        launch_reduce_y_fp8(yp, splits, Bs, s.A, sx, s.sL, y8, ty, nullptr, 1, st);
      else if (deq)
        launch_reduce_y_f16(yp, splits, Bs, s.A, sx, s.sL, y16, ty, nullptr, 1, st);
      else
        launch_reduce_y_bf16(yp, splits, Bs, s.A, yh, nullptr, st);
      check_launch(h, "reduce_y");
      launch_gemm2_tc(plan, EPI_APPLY, xp, nullptr, nullptr, wp, nullptr, h->d_status, st);
      check_launch(h, "gemm2_tc");
      LGW_TRY_CUDA(h, cudaStreamSynchronize(st));
      tc_plan_destroy(plan);
    } else {
      const int splits = gemm1_f64_splits(s, Bs);
      double *yp = wsT<double>(h, "yp64", (size_t)splits * Bs * s.A);
      launch_gemm1_f64(s, xp, Bs, yp, splits, st);
      check_launch(h, "gemm1_f64");
      launch_reduce_y_f64(yp, splits, Bs, s.A, Y64, st);
      check_launch(h, "reduce_y_f64");
      launch_gemm2_f64(s, Y64, Bs, EPI_APPLY, xp, nullptr, nullptr, wp, nullptr, st);
      check_launch(h, "gemm2_f64");
    }
    LGW_TRY_CUDA(h, cudaMemcpy2DAsync(Yo.dev, sizeof(double) * s.n_vc, wp, sizeof(double) * s.N,
                                      sizeof(double) * s.n_vc, n_vec, cudaMemcpyDeviceToDevice, st));
    Yo.finish(h);
    check_status(h);
  } catch (Fail &f) {
    return f.st;
  }
  return LGW_OK;
}

lgw_status lgw_lanczos_coeffs(lgw_handle *h, const lgw_system *sys, const lgw_problem *p,
                              const lgw_options *o, double *alpha, double *beta, double *beta0,
                              int32_t *k_eff) {
  lgw_status g = guard_handle(h);
  if (g != LGW_OK) return g;
  if (!sys || sys->h != h || !alpha || !beta || !beta0 || !k_eff)
    return set_err(h, LGW_ERR_ARG, "NULL argument to lgw_lanczos_coeffs");
  try {
    const SysDev &s = sys->s;
    cudaStream_t st = h->stream;
    LGW_TRY_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), st));
    Opts op = resolve_opts(h, o, s);
    ensure_copies(h, sys, op);
    ProbView pv = check_problem(h, s, p);
    OutBuf<double> a, b, b0;
    OutBuf<int32_t> ke;
    a.init(h, "out_alpha", alpha, (size_t)pv.B * op.k);
    b.init(h, "out_beta", beta, (size_t)pv.B * op.k);
    b0.init(h, "out_beta0", beta0, (size_t)pv.B);
    ke.init(h, "out_keff", k_eff, (size_t)pv.B);
    h->timing = false;
    run_lanczos(h, s, pv, op, a.dev, b.dev, b0.dev, ke.dev, nullptr, nullptr);
    a.finish(h);
    b.finish(h);
    b0.finish(h);
    ke.finish(h);
    check_status(h);
  } catch (Fail &f) {
    return f.st;
  }
  return LGW_OK;
}

lgw_status lgw_sigma_from_coeffs(lgw_handle *h, const lgw_system *sys, const lgw_problem *p,
                                 const lgw_options *o, const double *alpha, const double *beta,
                                 const double *beta0, const int32_t *k_eff, double *sigma,
                                 double *e_qp, double *z_qp) {
  lgw_status g = guard_handle(h);
  if (g != LGW_OK) return g;
  if (!sys || sys->h != h || !alpha || !beta || !beta0 || !k_eff)
    return set_err(h, LGW_ERR_ARG, "NULL argument to lgw_sigma_from_coeffs");
  try {
    const SysDev &s = sys->s;
    cudaStream_t st = h->stream;
    LGW_TRY_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), st));
    Opts op = resolve_opts(h, o, s);
    ProbView pv = check_problem(h, s, p);
    const double *da = in_dev(h, "in_alpha", alpha, (size_t)pv.B * op.k);
    const double *db = in_dev(h, "in_beta", beta, (size_t)pv.B * op.k);
    const double *db0 = in_dev(h, "in_beta0", beta0, (size_t)pv.B);
    const int *dke = in_dev(h, "in_keff", k_eff, (size_t)pv.B);
    OutBuf<double> sg, e, z;
    sg.init(h, "out_sigma", sigma, (size_t)pv.n_t * pv.n_freq * 2);
    e.init(h, "out_eqp", e_qp, (size_t)pv.n_t);
    z.init(h, "out_zqp", z_qp, (size_t)pv.n_t);
    h->timing = false;
    run_sigma(h, s, pv, op, da, db, db0, dke, sg.dev, e.dev, z.dev, nullptr, nullptr);
    sg.finish(h);
    e.finish(h);
    z.finish(h);
    check_status(h);
  } catch (Fail &f) {
    return f.st;
  }
  return LGW_OK;
}

lgw_status lgw_sigma_c(lgw_handle *h, const lgw_system *sys, const lgw_problem *p,
                       const lgw_options *o, double *sigma, double *e_qp, double *z_qp,
                       lgw_report *rep) {
  return sigma_c_impl(h, sys, p, o, nullptr, sigma, e_qp, z_qp, rep);
}

lgw_status lgw_sigma_c_tda(lgw_handle *h, const lgw_system *sys, const lgw_problem *p,
                           const lgw_options *o, double *sigma, double *e_qp, double *z_qp,
                           lgw_report *rep) {
  return sigma_c_impl(h, sys, p, o, nullptr, sigma, e_qp, z_qp, rep, true);
}

lgw_status lgw_sigma_offdiag(lgw_handle *h, const lgw_system *sys, const lgw_problem *p,
                             const lgw_options *o, int32_t n_pairs, const int32_t *pairs,
                             double *sigma_od) {
  lgw_status g = guard_handle(h);
  if (g != LGW_OK) return g;
  if (!sys || sys->h != h || n_pairs < 0 || (n_pairs > 0 && (!pairs || !sigma_od)))
    return set_err(h, LGW_ERR_ARG, "bad arguments to lgw_sigma_offdiag");
  try {
    const SysDev &s = sys->s;
    cudaStream_t st = h->stream;
    h->timing = false;
    LGW_TRY_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), st));
    Opts op = resolve_opts(h, o, s);
    ensure_copies(h, sys, op);
    ProbView pv = check_problem(h, s, p);
    if (n_pairs == 0) return LGW_OK;
    std::vector<int> hp = to_host(h, pairs, (size_t)2 * n_pairs);
    for (int x : hp)
      if (x < 0 || x >= pv.n_t) {
        set_err(h, LGW_ERR_SHAPE, "pair index %d outside [0, n_t = %d)", x, pv.n_t);
        throw Fail{LGW_ERR_SHAPE};
      }
    // virtual request: rows 2i, 2i+1 = factors of t + t' and t - t' (pair i)
    ProbView pv2 = pv;
    pv2.n_t = 2 * n_pairs;
    pv2.B = pv2.n_t * pv.n_m;
    pv2.targets.assign(pv2.n_t, 0);
    for (int i = 0; i < n_pairs; ++i) pv2.targets[2 * i] = pv2.targets[2 * i + 1] = pv.targets[hp[2 * i]];
    pv2.d_targets = in_dev(h, "od_targets", pv2.targets.data(), (size_t)pv2.n_t);
    const int *dpairs = in_dev(h, "od_pairs", hp.data(), hp.size());
    pv2.d_shift = nullptr;
    if (pv.d_M) {
      double *M2 = wsT<double>(h, "od_M", (size_t)pv2.B * s.n_aux);
      launch_pol_rows(pv.d_M, pv.n_m, s.n_aux, dpairs, n_pairs, M2, st);
      check_launch(h, "pol_rows");
      pv2.d_M = M2;
    } else {
      double *V2 = wsT<double>(h, "od_V", (size_t)pv2.B * s.n_vc);
      launch_pol_rows(pv.d_V, pv.n_m, s.n_vc, dpairs, n_pairs, V2, st);
      check_launch(h, "pol_rows");
      pv2.d_V = V2;
    }
    double *alpha = wsT<double>(h, "co_alpha", (size_t)pv2.B * op.k);
    double *beta = wsT<double>(h, "co_beta", (size_t)pv2.B * op.k);
    double *beta0 = wsT<double>(h, "co_beta0", (size_t)pv2.B);
    int *ke = wsT<int>(h, "co_keff", (size_t)pv2.B);
    double *sig2 = wsT<double>(h, "od_sigma", (size_t)pv2.n_t * pv.n_freq * 2);
    run_lanczos(h, s, pv2, op, alpha, beta, beta0, ke, nullptr, nullptr);
    run_sigma(h, s, pv2, op, alpha, beta, beta0, ke, sig2, nullptr, nullptr, nullptr, nullptr);
    OutBuf<double> out;
    out.init(h, "out_sigma_od", sigma_od, (size_t)n_pairs * pv.n_freq * 2);
    launch_pol_combine(sig2, n_pairs, pv.n_freq, out.dev, st);
    check_launch(h, "pol_combine");
    out.finish(h);
    check_status(h);
  } catch (Fail &f) {
    return f.st;
  }
  return LGW_OK;
}

lgw_status lgw_spectral_interval(lgw_handle *h, const lgw_system *sys, int32_t k, double *x_lo,
                                 double *x_hi) {
  lgw_status g = guard_handle(h);
  if (g != LGW_OK) return g;
  if (!sys || sys->h != h || !x_lo || !x_hi)
    return set_err(h, LGW_ERR_ARG, "NULL argument to lgw_spectral_interval");
  if (k < 1 || k > 4095) return set_err(h, LGW_ERR_ARG, "k = %d outside [1, 4095]", k);
  if (!sys->s.L64 && !sys->s.Lb)
    return set_err(h, LGW_ERR_UNSUPPORTED, "the interval needs the FP64 or the BF16 copy of L");
  try {
    LGW_TRY_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), h->stream));
    h->timing = false;
    estimate_interval(h, sys->s, k, *x_lo, *x_hi);
    check_status(h);
    if (k == 32) {   // the estimate lgw_sigma_c_poly uses when asked for one
      lgw_system *ms = const_cast<lgw_system *>(sys);
      ms->ivl_lo = *x_lo;
      ms->ivl_hi = *x_hi;
      ms->ivl_ok = true;
    }
  } catch (Fail &f) {
    return f.st;
  }
  return LGW_OK;
}

lgw_status lgw_sigma_band(lgw_handle *h, const lgw_system *sys, const lgw_problem *p,
                          const lgw_options *o, double *sigma, lgw_report *rep) {
  lgw_status g = guard_handle(h);
  if (g != LGW_OK) return g;
  if (!sys || sys->h != h || !sigma) return set_err(h, LGW_ERR_ARG, "bad arguments to lgw_sigma_band");
  try {
    const SysDev &s = sys->s;
    cudaStream_t st = h->stream;
    h->launches = 0;
    h->ev_used = 0;
    h->timing = rep != nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (rep) {
      std::memset(rep, 0, sizeof *rep);
      LGW_TRY_CUDA(h, cudaEventCreate(&t0));
      LGW_TRY_CUDA(h, cudaEventCreate(&t1));
      LGW_TRY_CUDA(h, cudaEventRecord(t0, st));
    }
    LGW_TRY_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), st));
    Opts op = resolve_opts(h, o, s);
    if (op.precision == LGW_FP8 || op.precision == LGW_FP8_DEQ) {
      set_err(h, LGW_ERR_UNSUPPORTED, "band Lanczos runs FP64 or BF16 contractions");
      throw Fail{LGW_ERR_UNSUPPORTED};
    }
    if (op.k > 512) {
      set_err(h, LGW_ERR_UNSUPPORTED, "band Lanczos: k = %d above its 512-step limit", op.k);
      throw Fail{LGW_ERR_UNSUPPORTED};
    }
    ensure_copies(h, sys, op);
    ProbView pv = check_problem(h, s, p);
    const int P = pv.n_t, G = pv.n_m, F = pv.n_freq, k = op.k;
    if (P < 1 || P > 8) {
      set_err(h, LGW_ERR_UNSUPPORTED, "band Lanczos: n_t = %d targets, 1..8 supported", P);
      throw Fail{LGW_ERR_UNSUPPORTED};
    }
    OutBuf<double> out;
    out.init(h, "out_sigma_band", sigma, (size_t)P * P * F * 2);
    double tacc[C_N] = {0};
    if (G > 0 && F > 0) {
      double *Tb = wsT<double>(h, "band_T", (size_t)G * k * (P + 1));
      double *R0 = wsT<double>(h, "band_R0", (size_t)G * P * P);
      int *keff = wsT<int>(h, "band_keff", (size_t)G);
      run_band(h, s, pv, op, Tb, R0, keff, rep ? tacc : nullptr);
      // polarisation vectors of the small problem: e_a, then e_a +- e_b
      const int nx = P + P * (P - 1);
      std::vector<double> xs((size_t)nx * P, 0.0);
      for (int a = 0; a < P; ++a) xs[(size_t)a * P + a] = 1.0;
      int q = 0;
      for (int a = 0; a < P; ++a)
        for (int b = a + 1; b < P; ++b, ++q) {
          double *xp = &xs[(size_t)(P + 2 * q) * P], *xm = xp + P;
          xp[a] = xm[a] = 1.0;
          xp[b] = 1.0;
          xm[b] = -1.0;
        }
      const double *dxs = in_dev(h, "band_xs", xs.data(), xs.size());
      const int Bx = nx * G;
      double *a2 = wsT<double>(h, "co_alpha", (size_t)Bx * k);
      double *b2 = wsT<double>(h, "co_beta", (size_t)Bx * k);
      double *b02 = wsT<double>(h, "co_beta0", (size_t)Bx);
      int *ke2 = wsT<int>(h, "co_keff", (size_t)Bx);
      double *scr = wsT<double>(h, "band_small", (size_t)Bx * (k + 2) * k);
      launch_band_small(Tb, R0, keff, G, k, P, dxs, nx, op.tol, scr, a2, b2, b02, ke2, st);
      check_launch(h, "band_small");
      ProbView pv3 = pv;
      pv3.n_t = nx;
      pv3.B = Bx;
      pv3.d_targets = nullptr;
      pv3.d_shift = nullptr;
      double *sigx = wsT<double>(h, "band_sigx", (size_t)nx * F * 2);
      run_sigma(h, s, pv3, op, a2, b2, b02, ke2, sigx, nullptr, nullptr, rep, tacc);
      launch_band_combine(sigx, P, F, out.dev, st);
      check_launch(h, "band_combine");
    } else if (out.dev) {
      LGW_TRY_CUDA(h, cudaMemsetAsync(out.dev, 0, sizeof(double) * (size_t)P * P * F * 2, st));
    }
    out.finish(h);
    if (rep) {
      LGW_TRY_CUDA(h, cudaEventRecord(t1, st));
      LGW_TRY_CUDA(h, cudaEventSynchronize(t1));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, t0, t1);
      cudaEventDestroy(t0);
      cudaEventDestroy(t1);
      rep->ms_total = ms;
      rep->ms_start = tacc[C_START];
      rep->ms_gemm1 = tacc[C_GEMM1];
      rep->ms_gemm2 = tacc[C_GEMM2];
      rep->ms_dots = tacc[C_DOTS];
      rep->ms_spectral = tacc[C_SPEC];
      rep->ms_cf = tacc[C_CF];
      rep->n_vectors = G;
      rep->gemm_flops = 4.0 * s.n_vc * (double)s.n_aux * (double)G * (double)k;
      rep->gpu_launches = h->launches;
      rep->k_min = rep->k_max = k;
    }
    check_status(h);
    h->timing = false;
  } catch (Fail &f) {
    h->timing = false;
    return f.st;
  }
  return LGW_OK;
}

lgw_status lgw_sigma_c_poly(lgw_handle *h, const lgw_system *sys, const lgw_problem *p,
                            const lgw_options *o, const lgw_poly *poly, double *sigma,
                            double *e_qp, double *z_qp, lgw_report *rep) {
  if (!poly) return h ? set_err(h, LGW_ERR_ARG, "polynomial descriptor is NULL") : LGW_ERR_ARG;
  return sigma_c_impl(h, sys, p, o, poly, sigma, e_qp, z_qp, rep);
}

lgw_status lgw_lanczos_coeffs_poly(lgw_handle *h, const lgw_system *sys, const lgw_problem *p,
                                   const lgw_options *o, const lgw_poly *pp, double *alpha,
                                   double *beta, double *beta0, int32_t *k_eff) {
  lgw_status g = guard_handle(h);
  if (g != LGW_OK) return g;
  if (!sys || sys->h != h || !pp || !alpha || !beta || !beta0 || !k_eff)
    return set_err(h, LGW_ERR_ARG, "NULL argument to lgw_lanczos_coeffs_poly");
  try {
    const SysDev &s = sys->s;
    cudaStream_t st = h->stream;
    LGW_TRY_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), st));
    Opts op = resolve_opts(h, o, s);
    ensure_copies(h, sys, op);
    PolyOp pstore;
    const PolyOp *poly = poly_arg(h, sys, pp, pstore);
    op.split = 0;
    op.split32 = 0;
    ProbView pv = check_problem(h, s, p);
    OutBuf<double> a, b, b0;
    OutBuf<int32_t> ke;
    a.init(h, "out_alpha", alpha, (size_t)pv.B * op.k);
    b.init(h, "out_beta", beta, (size_t)pv.B * op.k);
    b0.init(h, "out_beta0", beta0, (size_t)pv.B);
    ke.init(h, "out_keff", k_eff, (size_t)pv.B);
    h->timing = false;
    run_lanczos(h, s, pv, op, a.dev, b.dev, b0.dev, ke.dev, nullptr, nullptr, false, nullptr,
                poly);
    a.finish(h);
    b.finish(h);
    b0.finish(h);
    ke.finish(h);
    check_status(h);
  } catch (Fail &f) {
    return f.st;
  }
  return LGW_OK;
}

lgw_status lgw_sigma_c_batched(lgw_handle *h, int32_t n_sys, const lgw_system *const *systems,
                               const lgw_problem *problems, const lgw_options *o,
                               double *const *sigma, double *const *e_qp, double *const *z_qp,
                               lgw_report *rep) {
  lgw_status g = guard_handle(h);
  if (g != LGW_OK) return g;
  if (n_sys < 0 || (n_sys > 0 && (!systems || !problems || !sigma || !e_qp)))
    return set_err(h, LGW_ERR_ARG, "bad arguments to lgw_sigma_c_batched");
  for (int i = 0; i < n_sys; ++i)
    if (!systems[i] || systems[i]->h != h)
      return set_err(h, LGW_ERR_ARG, "bad system handle at index %d", i);
  if (rep) std::memset(rep, 0, sizeof *rep);
  if (n_sys == 0) return LGW_OK;
  const cudaStream_t caller = h->stream;
  // every exit restores the caller's stream and the default workspace names
  struct Restore {
    lgw_handle *h;
    cudaStream_t st;
    ~Restore() {
      h->stream = st;
      h->ws_prefix.clear();
      h->timing = false;
    }
  } restore{h, caller};
  try {
    h->launches = 0;
    h->ev_used = 0;
    h->timing = false;
    cudaEvent_t t0 = nullptr, t1 = nullptr, fork = nullptr;
    if (rep) {
      LGW_TRY_CUDA(h, cudaEventCreate(&t0));
      LGW_TRY_CUDA(h, cudaEventCreate(&t1));
      LGW_TRY_CUDA(h, cudaEventRecord(t0, caller));
    }
    LGW_TRY_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), caller));
    // systems are independent: up to 4 run at once, system i on lane i % 4
    const int S = std::min(n_sys, 4);
    while ((int)h->lanes.size() < S) {
      cudaStream_t l;
      LGW_TRY_CUDA(h, cudaStreamCreateWithFlags(&l, cudaStreamNonBlocking));
      h->lanes.push_back(l);
    }
    LGW_TRY_CUDA(h, cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    LGW_TRY_CUDA(h, cudaEventRecord(fork, caller));
    for (int l = 0; l < S; ++l) LGW_TRY_CUDA(h, cudaStreamWaitEvent(h->lanes[l], fork, 0));
    struct Done {
      int B, k, n_vc, n_aux, reorth;
      const int *ke;
    };
    std::vector<Done> done;
    for (int i = 0; i < n_sys; ++i) {
      const int lane = i % S;
      h->stream = h->lanes[lane];
      h->ws_prefix = "lane" + std::to_string(lane) + "/";
      const SysDev &s = systems[i]->s;
      Opts op = resolve_opts(h, o, s);
      ensure_copies(h, systems[i], op);
      ProbView pv = check_problem(h, s, &problems[i]);
      double *alpha = wsT<double>(h, "co_alpha", (size_t)std::max(1, pv.B) * op.k);
      double *beta = wsT<double>(h, "co_beta", (size_t)std::max(1, pv.B) * op.k);
      double *beta0 = wsT<double>(h, "co_beta0", (size_t)std::max(1, pv.B));
      int *ke = wsT<int>(h, "co_keff" + std::to_string(i), (size_t)std::max(1, pv.B));
      OutBuf<double> sg, e, z;
      sg.init(h, "out_sigma", sigma[i], (size_t)pv.n_t * pv.n_freq * 2);
      e.init(h, "out_eqp", e_qp[i], (size_t)pv.n_t);
      z.init(h, "out_zqp", z_qp ? z_qp[i] : nullptr, (size_t)pv.n_t);
      run_lanczos(h, s, pv, op, alpha, beta, beta0, ke, nullptr, nullptr);
      run_sigma(h, s, pv, op, alpha, beta, beta0, ke, sg.dev, e.dev, z.dev, nullptr, nullptr);
      sg.finish(h);
      e.finish(h);
      z.finish(h);
      done.push_back({pv.B, op.k, s.n_vc, s.n_aux, op.reorth, ke});
    }
    h->stream = caller;
    h->ws_prefix.clear();
    for (int l = 0; l < S; ++l) {
      LGW_TRY_CUDA(h, cudaEventRecord(fork, h->lanes[l]));
      LGW_TRY_CUDA(h, cudaStreamWaitEvent(caller, fork, 0));
    }
    cudaEventDestroy(fork);
    if (rep) {
      LGW_TRY_CUDA(h, cudaEventRecord(t1, caller));
      LGW_TRY_CUDA(h, cudaEventSynchronize(t1));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, t0, t1);
      cudaEventDestroy(t0);
      cudaEventDestroy(t1);
      rep->ms_total = ms;
      rep->gpu_launches = h->launches;
      int kmin = 1 << 30, kmax = 0;
      for (const Done &d : done) {
        std::vector<int> kv(d.B);
        if (d.B)
          LGW_TRY_CUDA(h, cudaMemcpy(kv.data(), d.ke, sizeof(int) * d.B, cudaMemcpyDeviceToHost));
        for (int x : kv) {
          kmin = std::min(kmin, x);
          kmax = std::max(kmax, x);
          if (d.reorth != LGW_REORTH_NONE)
            rep->reorth_elems += (double)d.n_vc * (double)x * (double)(x + 1) / 2.0;
        }
        rep->n_vectors += d.B;
        rep->gemm_flops += 4.0 * d.n_vc * (double)d.n_aux * (double)d.B * (double)d.k;
      }
      rep->k_min = rep->n_vectors ? kmin : 0;
      rep->k_max = kmax;
      rep->n_sub_batches = n_sys;
    }
    check_status(h);
  } catch (Fail &f) {
    return f.st;
  }
  return LGW_OK;
}

static lgw_status backward_impl(lgw_handle *h, const lgw_system *sys, const lgw_problem *p,
                                const lgw_options *o, const double *dE, double *dL,
                                double *deps, bool tda, const lgw_poly *pp = nullptr) {
  lgw_status g = guard_handle(h);
  if (g != LGW_OK) return g;
  if (!sys || sys->h != h || !dE) return set_err(h, LGW_ERR_ARG, "NULL argument to the backward call");
  try {
    cudaStream_t st = h->stream;
    h->timing = false;
    LGW_TRY_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), st));
    Opts op = resolve_opts(h, o, sys->s);
    ensure_copies(h, sys, op);
    const SysDev &s = tda ? tda_view(h, sys) : sys->s;
    if (op.qp_mode != 0) {
      set_err(h, LGW_ERR_UNSUPPORTED, "the adjoint differentiates the graphical QP solution (qp_mode 0)");
      throw Fail{LGW_ERR_UNSUPPORTED};
    }
    // FP64 contractions without reorthogonalisation: the exact reverse mode
    // of the three-term recurrence, recomputed from Krylov checkpoints;
    // otherwise the Krylov form over the stored basis
    const bool exact = op.reorth == LGW_REORTH_NONE && op.precision == LGW_FP64;
    const int ci = (o->ckpt_every > 0) ? o->ckpt_every : 16;
    if (o->ckpt_every < 0) {
      set_err(h, LGW_ERR_ARG, "ckpt_every < 0");
      throw Fail{LGW_ERR_ARG};
    }
    // the polynomial form is differentiated exactly only (the Krylov form
    // would need the eigenvectors of C behind p_g); its interval is held fixed
    PolyOp pstore;
    const PolyOp *poly = poly_arg(h, sys, pp, pstore);
    if (poly && !exact) {
      set_err(h, LGW_ERR_UNSUPPORTED,
              "the polynomial form's adjoint needs FP64 contractions without reorthogonalisation");
      throw Fail{LGW_ERR_UNSUPPORTED};
    }
    if (poly) {
      op.split = 0;
      op.split32 = 0;
    }
    // the adjoint contracts with the stored Krylov basis: FP64 (FP64 mode)
    // or the split float pair (BF16 mode with split arithmetic); the split
    // basis needs reorthogonalisation (otherwise the FP64 basis is kept)
    if (op.reorth == LGW_REORTH_NONE || op.precision == LGW_FP64) {
      op.split = 0;
      op.split32 = 0;
    }
    if (op.k > adj_max_k()) {
      set_err(h, LGW_ERR_UNSUPPORTED, "k = %d above the %d-step limit of the adjoint", op.k,
              adj_max_k());
      throw Fail{LGW_ERR_UNSUPPORTED};
    }
    if (!s.L64 || (op.precision != LGW_FP64 && !s.Ltb)) {
      set_err(h, LGW_ERR_UNSUPPORTED,
              "the adjoint needs the FP64 copy of L (and the BF16 copies for BF16/FP8)");
      throw Fail{LGW_ERR_UNSUPPORTED};
    }
    ProbView pv = check_problem(h, s, p);
    const int B = pv.B, k = op.k, N = s.N, A = s.A;
    const double *d_dE = in_dev(h, "in_dE", dE, (size_t)pv.n_t);
    OutBuf<double> oL, oe;
    oL.init(h, "out_dL", dL, (size_t)s.n_vc * s.n_aux);
    oe.init(h, "out_deps", deps, (size_t)(s.n_v + s.n_c));
    double *gdeps = wsT<double>(h, "adj_deps", (size_t)(s.n_v + s.n_c));
    LGW_TRY_CUDA(h, cudaMemsetAsync(gdeps, 0, sizeof(double) * (s.n_v + s.n_c), st));
    if (B == 0 || pv.n_t == 0) {
      if (oL.dev) LGW_TRY_CUDA(h, cudaMemsetAsync(oL.dev, 0, sizeof(double) * s.n_vc * s.n_aux, st));
      if (pv.n_t > 0) {
        // no summed orbitals: E_t = eps_t + s_t, Z_t = 1
        std::vector<double> one(pv.n_t, 1.0);
        double *Z1 = wsT<double>(h, "adj_Z", (size_t)pv.n_t);
        LGW_TRY_CUDA(h, cudaMemcpyAsync(Z1, one.data(), sizeof(double) * pv.n_t,
                                        cudaMemcpyHostToDevice, st));
        double *dD = wsT<double>(h, "adj_dDelta", (size_t)N);
        LGW_TRY_CUDA(h, cudaMemsetAsync(dD, 0, sizeof(double) * N, st));
        launch_adj_deps(dD, s.n_v, s.n_c, pv.d_targets, pv.n_t, Z1, d_dE, gdeps, st);
        check_launch(h, "adj_deps");
      }
      if (oe.dev)
        LGW_TRY_CUDA(h, cudaMemcpyAsync(oe.dev, gdeps, sizeof(double) * (s.n_v + s.n_c),
                                        cudaMemcpyDeviceToDevice, st));
      oL.finish(h);
      oe.finish(h);
      LGW_TRY_CUDA(h, cudaStreamSynchronize(st));
      return LGW_OK;
    }
    const bool tc = op.precision != LGW_FP64;
    // sub-batch: the caller's b_sub, else as many vectors as fit in half of
    // the free device memory (plus what the handle already holds)
    {
      size_t fr = 0, tot = 0;
      LGW_TRY_CUDA(h, cudaMemGetInfo(&fr, &tot));
      size_t held = 0;
      for (auto &kv : h->bufs) held += kv.second.n;
      const int cs = std::min(ci, k), nseg = (k + ci - 1) / ci;
      // exact form: checkpoints, the recomputation window, ubar_j, the qbar ring
      // and row buffers, plus (polynomial form) Clenshaw's 2 g + 1 vectors
      const int gp = poly ? poly->g : 0;
      const double per_vec =
          exact ? 8.0 * (2 * nseg + 2 * cs + 12 + 2 * gp + 1) * N + 16.0 * (cs + gp) * A +
                      40.0 * k * k
                : 8.0 * (k + 1) * N + (tc ? 4.0 * k * N : 0.0) + 20.0 * k * A + 48.0 * N +
                      40.0 * k * k;
      const double budget = 0.5 * (double)(fr + held);
      int fit = (int)std::min<double>(budget / per_vec, 1 << 20);
      fit = std::max(PAD_VEC, fit / PAD_VEC * PAD_VEC);
      if (op.b_sub <= 0) op.b_sub = std::min(B, fit);
    }
    const int bsub = std::min(op.b_sub, B);
    const bool one_pass = bsub >= B;
    if (tc && !sys->Ltb_lo) {
      lgw_system *ms = const_cast<lgw_system *>(sys);
      LGW_TRY_CUDA(h, cudaMalloc(&ms->Ltb_lo, sizeof(__nv_bfloat16) * (size_t)N * A));
      launch_split_t(BasisRef{s.L64, nullptr, nullptr}, N, A, A, nullptr, ms->Ltb_lo, st);
      check_launch(h, "split_t(L lo)");
    }
    // coefficients of the forward pass
    double *alpha = wsT<double>(h, "co_alpha", (size_t)B * k);
    double *beta = wsT<double>(h, "co_beta", (size_t)B * k);
    double *beta0 = wsT<double>(h, "co_beta0", (size_t)B);
    int *ke = wsT<int>(h, "co_keff", (size_t)B);
    double *E = wsT<double>(h, "adj_E", (size_t)pv.n_t);
    double *Z = wsT<double>(h, "adj_Z", (size_t)pv.n_t);
    // accumulators
    double *SC = wsT<double>(h, "adj_SC", (size_t)N * A);
    double *SB = pv.d_M ? wsT<double>(h, "adj_SB", (size_t)N * s.n_aux) : nullptr;
    double *dD = wsT<double>(h, "adj_dDelta", (size_t)N);
    LGW_TRY_CUDA(h, cudaMemsetAsync(SC, 0, sizeof(double) * N * A, st));
    if (SB) LGW_TRY_CUDA(h, cudaMemsetAsync(SB, 0, sizeof(double) * N * s.n_aux, st));
    LGW_TRY_CUDA(h, cudaMemsetAsync(dD, 0, sizeof(double) * N, st));

    auto forward_sigma = [&]() {
      run_sigma(h, s, pv, op, alpha, beta, beta0, ke, nullptr, E, Z, nullptr, nullptr,
                poly ? 1 : (tda ? 2 : 0));
    };
    // Krylov checkpoints of the exact mode: (q_{s0-1}, q_s0) at every segment
    // start s0 = 0, ci, 2 ci, ... (q_{-1} = 0), copied out of the forward's
    // three-vector ring
    const int nseg = (k + ci - 1) / ci;
    double *ckpt = nullptr;
    StepHook keep_ckpt = [&](const VecCtx &c, int j) {
      const size_t BN = (size_t)c.Bs * c.N;
      if (j < 0) {
        ckpt = wsT<double>(h, "rev_ckpt", (size_t)nseg * 2 * BN);
        LGW_TRY_CUDA(h, cudaMemsetAsync(ckpt, 0, sizeof(double) * BN, st));
        LGW_TRY_CUDA(h, cudaMemcpyAsync(ckpt + BN, slot_ptr(c, 0), sizeof(double) * BN,
                                        cudaMemcpyDeviceToDevice, st));
        return;
      }
      const int nx = j + 1;
      if (nx % ci != 0 || nx >= k) return;
      double *dst = ckpt + (size_t)(nx / ci) * 2 * BN;
      LGW_TRY_CUDA(h, cudaMemcpyAsync(dst, slot_ptr(c, j), sizeof(double) * BN,
                                      cudaMemcpyDeviceToDevice, st));
      LGW_TRY_CUDA(h, cudaMemcpyAsync(dst + BN, slot_ptr(c, nx), sizeof(double) * BN,
                                      cudaMemcpyDeviceToDevice, st));
    };
    SubBatchHook adjoint = [&](const VecCtx &c) {
      if (one_pass) forward_sigma();
      const int Bs = c.Bs;
      const BasisRef qb = op.split ? BasisRef{nullptr, c.bhi, c.blo}
                                   : BasisRef{c.basis, nullptr, nullptr};
      AdjCtx a{};
      a.N = N;
      a.Bs = Bs;
      a.nvec = c.nvec;
      a.vec0 = c.vec0;
      a.k = k;
      a.n_m = pv.n_m;
      a.n_v = s.n_v;
      a.alpha = alpha;
      a.beta = beta;
      a.beta0 = beta0;
      a.k_eff = ke;
      a.E = E;
      a.Z = Z;
      a.dE = d_dE;
      a.eps = s.eps;
      a.m_idx = pv.d_m_idx;
      a.delta = pv.delta;
      const size_t kk = (size_t)k * k;
      a.theta = wsT<double>(h, "adj_theta", (size_t)Bs * k);
      a.V = wsT<double>(h, "adj_V", (size_t)Bs * kk);
      a.Phi = wsT<double>(h, "adj_Phi", (size_t)Bs * kk);
      a.X = wsT<double>(h, "adj_X", (size_t)Bs * kk);
      a.ay = wsT<double>(h, "adj_ay", (size_t)Bs * k);
      a.Gam = wsT<double>(h, "adj_Gam", (size_t)Bs * kk);
      a.Gamf = tc ? wsT<float>(h, "adj_Gamf", (size_t)Bs * kk) : nullptr;
      a.dz = wsT<double>(h, "adj_dz", (size_t)Bs);
      a.status = h->d_status;
      a.tda = tda ? 1 : 0;
      a.poly = poly ? 1 : 0;
      launch_eig_full(a, st);
      check_launch(h, "eig_full");
      launch_adj_coeffs(a, st);
      check_launch(h, "adj_coeffs");
      if (exact) {
        reverse_sweep(h, s, pv, op, c, a, ckpt, ci, SC, SB, dD, gdeps, poly);
        return;
      }
      double *Y = wsT<double>(h, "adj_Y", (size_t)Bs * N);
      double *Gd = wsT<double>(h, "adj_Gd", (size_t)Bs * N);
      if (tc)
        launch_adj_rows_f32(a, qb, Y, Gd, st);
      else
        launch_adj_rows(a, qb, Y, Gd, st);
      check_launch(h, "adj_rows");
      const int rows = k * Bs;
      double *P = wsT<double>(h, "adj_P", (size_t)rows * A);
      double *R = wsT<double>(h, "adj_R", (size_t)rows * A);
      if (tc) {
        // P = Q^T D L: three split-BF16 products, FP64 sums of 16384-long chunks
        __nv_bfloat16 *Shi = wsT<__nv_bfloat16>(h, "adj_Shi", (size_t)rows * N);
        __nv_bfloat16 *Slo = wsT<__nv_bfloat16>(h, "adj_Slo", (size_t)rows * N);
        __nv_bfloat16 *Rhi = wsT<__nv_bfloat16>(h, "adj_Rhi", (size_t)rows * A);
        __nv_bfloat16 *Rlo = wsT<__nv_bfloat16>(h, "adj_Rlo", (size_t)rows * A);
        char err[256];
        launch_split_scaled(qb, rows, N, s.dsq, Shi, Slo, st);
        check_launch(h, "split_scaled(D Q)");
        // Ltb is K-block-major; the adjoint's own Ltb_lo is row-major
        const __nv_bfloat16 *pa[3] = {s.Ltb, s.Ltb, sys->Ltb_lo};
        const int pk[3] = {1, 1, 0};
        const __nv_bfloat16 *pb[3] = {Shi, Slo, Shi};
        if (!tc_gemm_f64out(3, pa, pk, pb, A, rows, N, 16384, P, A, 0, h->d_status, st, err,
                            sizeof err)) {
          set_err(h, LGW_ERR_CUDA, "%s", err);
          throw Fail{LGW_ERR_CUDA};
        }
        check_launch(h, "tc_gemm_f64out(P)");
        launch_gamma_p(a, P, A, R, st);
        check_launch(h, "gamma_p");
        // SC += Q R  (M = N_aux, N = N_vc, K = k Bs, transposed split operands)
        launch_split_t(BasisRef{R, nullptr, nullptr}, rows, A, A, Rhi, Rlo, st);
        check_launch(h, "split_t(R)");
        launch_split_t(qb, rows, N, N, Shi, Slo, st);
        check_launch(h, "split_t(Q)");
        const __nv_bfloat16 *qa[3] = {Rhi, Rhi, Rlo};
        const __nv_bfloat16 *qb[3] = {Shi, Slo, Shi};
        if (!tc_gemm_f64out(3, qa, nullptr, qb, A, N, rows, 16384, SC, A, 1, h->d_status, st, err,
                            sizeof err)) {
          set_err(h, LGW_ERR_CUDA, "%s", err);
          throw Fail{LGW_ERR_CUDA};
        }
        check_launch(h, "tc_gemm_f64out(SC)");
      } else {
        // P = Q^T D L over the k * Bs basis rows (FP64 GEMM1), R = Gam P
        const int sp = gemm1_f64_splits(s, rows);
        double *Pp = sp > 1 ? wsT<double>(h, "adj_Pp", (size_t)sp * rows * A) : P;
        launch_gemm1_f64(s, c.basis, rows, Pp, sp, st);
        check_launch(h, "gemm1_f64(adjoint)");
        if (sp > 1) {
          launch_reduce_y_f64(Pp, sp, rows, A, P, st);
          check_launch(h, "reduce_y_f64(adjoint)");
        }
        launch_gamma_p(a, P, A, R, st);
        check_launch(h, "gamma_p");
        launch_atb_f64(c.basis, N, R, A, rows, N, A, SC, st);
        check_launch(h, "atb_f64(SC)");
      }
      // SB += Y^T M
      if (SB) {
        launch_atb_f64(Y, N, pv.d_M + (size_t)c.vec0 * s.n_aux, s.n_aux, c.nvec, N, s.n_aux, SB,
                       st);
        check_launch(h, "atb_f64(SB)");
      }
      launch_adj_accumulate(a, s.Delta, qb, Y, Gd, dD, gdeps, st);
      check_launch(h, "adj_accumulate");
    };
    // the exact mode keeps only the three-vector ring and the checkpoints
    const bool keep = !exact;
    const StepHook *sh = exact ? &keep_ckpt : nullptr;
    if (one_pass) {
      run_lanczos(h, s, pv, op, alpha, beta, beta0, ke, nullptr, nullptr, keep, &adjoint, poly,
                  sh);
    } else {
      run_lanczos(h, s, pv, op, alpha, beta, beta0, ke, nullptr, nullptr, false, nullptr, poly);
      forward_sigma();
      run_lanczos(h, s, pv, op, alpha, beta, beta0, ke, nullptr, nullptr, keep, &adjoint, poly,
                  sh);
    }
    double *dLdev = oL.dev ? oL.dev : wsT<double>(h, "adj_dL", (size_t)s.n_vc * s.n_aux);
    // the exact mode accumulates SC = sum_j (ubar_j y_j^T + q_j ybar_j^T) = 2 G D L
    launch_adj_dL(s.L64, s.dsq, SC, SB, A, s.n_vc, s.n_aux, exact ? 0.5 * s.kf : s.kf, dLdev, dD,
                  tda ? 1 : 0, st);
    check_launch(h, "adj_dL");
    launch_adj_deps(dD, s.n_v, s.n_c, pv.d_targets, pv.n_t, Z, d_dE, gdeps, st);
    check_launch(h, "adj_deps");
    if (oe.dev)
      LGW_TRY_CUDA(h, cudaMemcpyAsync(oe.dev, gdeps, sizeof(double) * (s.n_v + s.n_c),
                                      cudaMemcpyDeviceToDevice, st));
    oL.finish(h);
    oe.finish(h);
    check_status(h);
  } catch (Fail &f) {
    return f.st;
  }
  return LGW_OK;
}

lgw_status lgw_sigma_c_backward(lgw_handle *h, const lgw_system *sys, const lgw_problem *p,
                                const lgw_options *o, const double *dE, double *dL,
                                double *deps) {
  return backward_impl(h, sys, p, o, dE, dL, deps, false);
}

lgw_status lgw_sigma_c_tda_backward(lgw_handle *h, const lgw_system *sys, const lgw_problem *p,
                                    const lgw_options *o, const double *dE, double *dL,
                                    double *deps) {
  return backward_impl(h, sys, p, o, dE, dL, deps, true);
}

lgw_status lgw_sigma_c_poly_backward(lgw_handle *h, const lgw_system *sys, const lgw_problem *p,
                                     const lgw_options *o, const lgw_poly *poly, const double *dE,
                                     double *dL, double *deps) {
  if (!poly) return set_err(h, LGW_ERR_ARG, "NULL polynomial to lgw_sigma_c_poly_backward");
  return backward_impl(h, sys, p, o, dE, dL, deps, false, poly);
}

lgw_status lgw_sigma_x(lgw_handle *h, const lgw_system *sys, const lgw_problem *p,
                       double *sigma_x) {
  lgw_status g = guard_handle(h);
  if (g != LGW_OK) return g;
  if (!sys || sys->h != h || !sigma_x) return set_err(h, LGW_ERR_ARG, "NULL argument to lgw_sigma_x");
  try {
    const SysDev &s = sys->s;
    cudaStream_t st = h->stream;
    LGW_TRY_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), st));
    ProbView pv = check_problem(h, s, p);
    if (!pv.d_M) {
      set_err(h, LGW_ERR_UNSUPPORTED, "the exchange self-energy needs the pair factors M");
      throw Fail{LGW_ERR_UNSUPPORTED};
    }
    OutBuf<double> out;
    out.init(h, "out_sigma_x", sigma_x, (size_t)pv.n_t);
    launch_sigma_x(pv.d_M, pv.n_t, pv.n_m, s.n_aux, pv.d_m_idx, s.n_v, out.dev, st);
    if (pv.n_t > 0) check_launch(h, "sigma_x");
    out.finish(h);
    check_status(h);
  } catch (Fail &f) {
    return f.st;
  }
  return LGW_OK;
}

lgw_status lgw_fit_factors(lgw_handle *h, int32_t n_pairs, int32_t n_aux, const double *C,
                           const double *metric, double *B) {
  lgw_status g = guard_handle(h);
  if (g != LGW_OK) return g;
  if (n_pairs < 0 || n_aux < 1 || (n_pairs > 0 && (!C || !B)) || !metric)
    return set_err(h, LGW_ERR_ARG, "bad arguments to lgw_fit_factors");
  try {
    cudaStream_t st = h->stream;
    LGW_TRY_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), st));
    const double *Vd = in_dev(h, "in_metric", metric, (size_t)n_aux * n_aux);
    double *R = wsT<double>(h, "fit_R", (size_t)n_aux * n_aux);
    LGW_TRY_CUDA(h, cudaMemcpyAsync(R, Vd, sizeof(double) * n_aux * n_aux,
                                    cudaMemcpyDeviceToDevice, st));
    h->launches += launch_cholesky(R, n_aux, h->d_status, st);
    check_launch(h, "cholesky");
    if (n_pairs > 0) {
      const double *Cd = in_dev(h, "in_fitC", C, (size_t)n_pairs * n_aux);
      OutBuf<double> out;
      out.init(h, "out_fitB", B, (size_t)n_pairs * n_aux);
      launch_gemm_nn_f64(Cd, R, n_pairs, n_aux, n_aux, out.dev, st);
      check_launch(h, "gemm_nn_f64");
      out.finish(h);
    }
    check_status(h);
  } catch (Fail &f) {
    return f.st;
  }
  return LGW_OK;
}

}  // extern "C"

// ===========================================================================
// Allocation-free variant of lgw_sigma_from_coeffs.
//
// Some callers cannot let a library allocate device memory while they run:
// services that hand the library a fixed device-memory budget at start-up,
// or latency-bound loops where cudaMalloc/cudaFree would synchronise the
// device and stall other streams.  This entry point performs the spectral
// map, the continued fractions on the grid and the QP solve with all of its
// scratch in one file-scope device array of fixed size; the caller passes
// inputs and outputs as device pointers.
// ===========================================================================
namespace {

// 2^21 doubles = 16 MiB on every device that loads the library, held until
// the process exits.  Layout per call: Jacobi a [B][k], b2 [B][k], w0 [B],
// depth [B] (ints, rounded up), three tridiagonal work rows [3][B][k], one
// word for the smallest Gauss node.
constexpr size_t kNoallocDoubles = (size_t)1 << 21;
static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_addr[kMaxDevices] = {nullptr};

// Sets the Gauss-node minimum word and checks every target / summed index
// and every depth k_eff against [0, k].  It only reads the index arrays;
// the caller reads the status word before launching anything that
// dereferences an index.
__global__ void k_noalloc_prologue(unsigned long long *min_theta_bits, const int *targets, int n_t,
                                   const int *m_idx, int n_m, int norb, const int *k_eff, int B,
                                   int k, unsigned *status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *min_theta_bits = 0x7FEFFFFFFFFFFFFFull;   // largest finite double
  if (i < n_t && (targets[i] < 0 || targets[i] >= norb)) atomicOr(status, ST_BAD_INPUT);
  if (i < n_m && (m_idx[i] < 0 || m_idx[i] >= norb)) atomicOr(status, ST_BAD_INPUT);
  if (i < B && (k_eff[i] < 0 || k_eff[i] > k)) atomicOr(status, ST_BAD_INPUT);
}

// Device memory of device `dev` (managed memory counts as any device's).
bool is_device_ptr_on(const void *p, int dev) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

size_t noalloc_doubles_needed(size_t B, size_t k) {
  return 2 * B * k + B + (B + 1) / 2 + 3 * B * k + 1;
}

}  // namespace

extern "C" lgw_status lgw_sigma_from_coeffs_noalloc(lgw_handle *h, const lgw_system *sys,
                                                    const lgw_problem *p, const lgw_options *o,
                                                    const double *alpha, const double *beta,
                                                    const double *beta0, const int32_t *k_eff,
                                                    double *sigma, double *e_qp, double *z_qp) {
  lgw_status g = guard_handle(h);
  if (g != LGW_OK) return g;
  if (!sys || sys->h != h || !p || !o || !alpha || !beta || !beta0 || !k_eff || !sigma ||
      !e_qp)
    return set_err(h, LGW_ERR_ARG, "NULL argument to lgw_sigma_from_coeffs_noalloc");
  const SysDev &s = sys->s;
  const int n_t = p->n_t, n_m = p->n_m, n_freq = p->n_freq, k = o->k;
  if (n_t < 1 || n_m < 1 || n_freq < 1 || !p->targets || !p->m_idx || !p->omega)
    return set_err(h, LGW_ERR_ARG, "noalloc: n_t, n_m, n_freq must be >= 1 with their arrays");
  if (k < 1 || k > s.n_vc) return set_err(h, LGW_ERR_ARG, "noalloc: k outside [1, n_vc]");
  if (k > 4095)
    return set_err(h, LGW_ERR_UNSUPPORTED, "noalloc: k = %d above the 4095-step limit", k);
  if (o->qp_mode != 0 && o->qp_mode != 1)
    return set_err(h, LGW_ERR_ARG, "noalloc: unknown qp_mode %d", o->qp_mode);
  if (!(p->delta > 0.0)) return set_err(h, LGW_ERR_ARG, "noalloc: delta must be > 0");
  const void *dev_ptrs[] = {alpha, beta, beta0, k_eff, sigma, e_qp, p->targets, p->m_idx,
                            p->omega};
  for (const void *q : dev_ptrs)
    if (!is_device_ptr_on(q, h->device))
      return set_err(h, LGW_ERR_ARG, "noalloc: every array must be device memory of device %d",
                     h->device);
  if ((z_qp && !is_device_ptr_on(z_qp, h->device)) ||
      (p->static_shift && !is_device_ptr_on(p->static_shift, h->device)))
    return set_err(h, LGW_ERR_ARG, "noalloc: every array must be device memory of device %d",
                   h->device);
  const size_t B = (size_t)n_t * (size_t)n_m;
  if (noalloc_doubles_needed(B, (size_t)k) > kNoallocDoubles)
    return set_err(h, LGW_ERR_UNSUPPORTED,
                   "noalloc: n_t*n_m*(5k+2) exceeds the %zu-double static scratch (B=%zu, k=%d)",
                   kNoallocDoubles, B, k);
  if (h->device < 0 || h->device >= kMaxDevices)
    return set_err(h, LGW_ERR_UNSUPPORTED, "noalloc: device index beyond %d", kMaxDevices);

  // One-time set-up per device: host code cannot use the array's name as a
  // device address, so fetch the address with that device current.
  double *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[h->device]) {
      void *ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess)
        return set_err(h, LGW_ERR_CUDA, "noalloc: cudaGetSymbolAddress failed: %s",
                       cudaGetErrorString(e));
      g_noalloc_addr[h->device] = static_cast<double *>(ptr);
    }
    base = g_noalloc_addr[h->device];
  }
  JacobiBufs jb;
  jb.a = base;
  jb.b2 = jb.a + B * k;
  jb.w0 = jb.b2 + B * k;
  jb.n = reinterpret_cast<int *>(jb.w0 + B);
  double *work = jb.w0 + B + (B + 1) / 2;
  unsigned long long *mt = reinterpret_cast<unsigned long long *>(work + 3 * B * k);

  cudaStream_t st = h->stream;
  if (cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), st) != cudaSuccess)
    return set_err(h, LGW_ERR_CUDA, "noalloc: status reset failed");
  // Index check first, and its verdict read back before any kernel that
  // dereferences an index (eps[m], eps[t], the k_eff-deep rows) is queued.
  const size_t nmax = std::max<size_t>(std::max(n_t, n_m), B);
  k_noalloc_prologue<<<(unsigned)((nmax + 255) / 256), 256, 0, st>>>(
      mt, p->targets, n_t, p->m_idx, n_m, s.n_v + s.n_c, k_eff, (int)B, k, h->d_status);
  {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
      return set_err(h, LGW_ERR_CUDA, "noalloc: index check launch failed: %s",
                     cudaGetErrorString(e));
    unsigned stw = 0;
    if (cudaMemcpyAsync(&stw, h->d_status, sizeof stw, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return set_err(h, LGW_ERR_CUDA, "noalloc: status read failed");
    if (stw & ST_BAD_INPUT)
      return set_err(h, LGW_ERR_SHAPE,
                     "noalloc: orbital index outside [0, n_v + n_c) or k_eff outside [0, k]");
  }
  launch_spectral_impl(alpha, beta, beta0, k_eff, (int)B, k, jb, work, mt, h->d_status, st);
  CfProblem cp{};
  cp.n_t = n_t;
  cp.n_m = n_m;
  cp.n_freq = n_freq;
  cp.k = k;
  cp.targets = p->targets;
  cp.m_idx = p->m_idx;
  cp.eps = s.eps;
  cp.n_v = s.n_v;
  cp.omega = p->omega;
  cp.delta = p->delta;
  cp.shift = p->static_shift;
  cp.qp_mode = o->qp_mode;
  launch_cf_grid(cp, jb, sigma, nullptr, 1, st);
  const int qp_iter = o->qp_max_iter > 0 ? o->qp_max_iter : 50;
  const double qp_tol = o->qp_tol > 0 ? o->qp_tol : 1e-10;
  launch_qp(cp, jb, sigma, qp_iter, qp_tol, e_qp, z_qp, h->d_status, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return set_err(h, LGW_ERR_CUDA, "noalloc: kernel launch failed: %s", cudaGetErrorString(e));
  unsigned stw = 0;
  if (cudaMemcpyAsync(&stw, h->d_status, sizeof stw, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return set_err(h, LGW_ERR_CUDA, "noalloc: status read failed");
  if (stw & ST_TIMEOUT) return set_err(h, LGW_ERR_TIMEOUT, "a bounded device wait ran out");
  if (stw & ST_NOT_SPD) return set_err(h, LGW_ERR_NOT_SPD, "non-positive Gauss node");
  if (stw & ST_NO_CONV)
    return set_err(h, LGW_ERR_NO_CONVERGENCE, "tridiagonal eigensolver or QP did not converge");
  return LGW_OK;
}
