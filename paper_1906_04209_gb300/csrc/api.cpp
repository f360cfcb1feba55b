// C ABI of the narrow capture / narrow escape solver (see include/ncs.h).
// Host orchestration only: every step of the matrix-vector product and of the
// Krylov iteration runs in the CUDA kernels of kernels.cu, tree.cu and blas.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <atomic>
#include <chrono>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.hpp"
#include "numerics.hpp"
#ifdef _OPENMP
#include <omp.h>
#endif

using ncs::DeviceData;

namespace ncs {
std::atomic<long long> g_launches{0};
}  // namespace ncs

namespace {

const char* g_static_err = "ncs: no context";

struct Fail {
  int code;
  std::string msg;
};

#define CU(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) throw Fail{e_ == cudaErrorMemoryAllocation ? NCS_E_OOM : NCS_E_CUDA, \
                                      std::string(#call) + ": " + cudaGetErrorString(e_)};    \
  } while (0)

int log_level() {
  static int lv = -1;
  if (lv < 0) {
    const char* e = std::getenv("NCS_LOG");
    lv = e ? std::atoi(e) : 0;
  }
  return lv;
}

template <typename T>
void dev_free(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

template <typename T>
T* dev_upload(const std::vector<T>& h) {
  T* p = nullptr;
  CU(cudaMalloc(&p, std::max<size_t>(1, h.size()) * sizeof(T)));
  if (!h.empty()) CU(cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return p;
}

template <typename T>
T* dev_alloc(size_t n) {
  T* p = nullptr;
  CU(cudaMalloc(&p, std::max<size_t>(1, n) * sizeof(T)));
  return p;
}

// The captured Arnoldi steps hold the layout's, the workspace's and the product path's
// pointers: dropped whenever one of them changes.
void invalidate_graphs(ncs_ctx* c) {
  for (int p = 0; p < ncs_ctx::kGraphSlots; ++p)
    if (c->step_graph[p]) {
      cudaGraphExecDestroy(c->step_graph[p]);
      c->step_graph[p] = nullptr;
      c->step_graph_kernels[p] = 0;
    }
}

void free_krylov(ncs_ctx* c) {
  invalidate_graphs(c);
  dev_free(c->V);
  dev_free(c->work);
  dev_free(c->partial);
  dev_free(c->hdev);
  dev_free(c->gmem);
  c->gd = ncs::GmresDev();
  if (c->st_host) cudaFreeHost(c->st_host);
  c->st_host = nullptr;
  c->Vcap = 0;
}

// Both trees (the product's and the mixed solve's inner one), host and device.
void drop_trees(ncs_ctx* c) {
  ncs::tree_free(c->tdev);
  ncs::tree_free(c->tdev_in);
  c->tree_built = c->tree_uploaded = false;
  c->tree_in_built = c->tree_in_uploaded = false;
  c->tree = ncs::TreeHost();
  c->tree_in = ncs::TreeHost();
}

void free_layout(ncs_ctx* c) {
  DeviceData& d = c->d;
  dev_free(d.centres);
  dev_free(d.soff64);
  dev_free(d.soff32);
  dev_free(d.rho64);
  dev_free(d.rho32);
  dev_free(d.z);
  dev_free(d.Apack);
  free_krylov(c);
  drop_trees(c);
  d.N = 0;
}

void free_all(ncs_ctx* c) {
  free_layout(c);
  DeviceData& d = c->d;
  dev_free(d.zloc);
  dev_free(d.sloc);
  dev_free(d.TT64);
  dev_free(d.TT32);
  dev_free(d.PT64);
  dev_free(d.PT32);
  dev_free(d.I);
  dev_free(d.rep_p);
  dev_free(d.rep_off);
  dev_free(d.rep_rho);
  dev_free(d.logtab);
  dev_free(d.Tpack);
  dev_free(d.Ppack);
  dev_free(d.tc_err);
  dev_free(c->near_d);
  dev_free(c->near_i);
  c->near_ready = false;
  if (c->stream) cudaStreamDestroy(c->stream);
  c->stream = nullptr;
}

// Uploads the precompute: all outgoing representations stacked (T_k transposed into one
// K x p_total matrix, skeleton offsets), P transposed, Zernike-node offsets, I.
void upload_operator(ncs_ctx* c) {
  const ncs::Precomputed& pc = c->pc;
  DeviceData& d = c->d;
  d.K = pc.K;
  d.Kstar = pc.Kstar;
  const int nrep = (int)pc.reps.size();
  std::vector<int> rp(nrep), ro(nrep);
  std::vector<double> rr(nrep);
  int pt = 0, pmax = 0;
  for (int r = 0; r < nrep; ++r) {
    rp[r] = pc.reps[r].p;
    ro[r] = pt;
    rr[r] = pc.reps[r].rho_min;
    pt += rp[r];
    pmax = std::max(pmax, rp[r]);
  }
  d.p = pt;
  d.pmax = pmax;
  d.p0 = rp[0];
  d.nrep = nrep;
  std::vector<double> TT((size_t)pc.K * pt), sl(3 * (size_t)pt), PT((size_t)pc.Kstar * pc.K);
  for (int r = 0; r < nrep; ++r)
    for (int m = 0; m < rp[r]; ++m) {
      for (int k = 0; k < pc.K; ++k) TT[(size_t)k * pt + ro[r] + m] = pc.reps[r].T[(size_t)m * pc.K + k];
      for (int a = 0; a < 3; ++a) sl[3 * (size_t)(ro[r] + m) + a] = pc.reps[r].sloc[3 * (size_t)m + a];
    }
  for (int j = 0; j < pc.K; ++j)
    for (int q = 0; q < pc.Kstar; ++q) PT[(size_t)q * pc.K + j] = pc.P[(size_t)j * pc.Kstar + q];
  std::vector<float> TT32(TT.begin(), TT.end()), PT32(PT.begin(), PT.end());
  std::vector<float> T32((size_t)pt * pc.K);
  for (int r = 0; r < nrep; ++r)
    for (int m = 0; m < rp[r]; ++m)
      for (int k = 0; k < pc.K; ++k) T32[(size_t)(ro[r] + m) * pc.K + k] = (float)pc.reps[r].T[(size_t)m * pc.K + k];
  std::vector<float> P32(pc.P.begin(), pc.P.end());
  {
    // tensor-core operands: TF32 hi/lo blocks packed once on the device
    float* T32d = dev_upload(T32);
    float* P32d = dev_upload(P32);
    d.Tpack = dev_alloc<uint32_t>((size_t)ncs::tc_pack_words(pt, pc.K, ncs::tc_block_cols(pt)));
    d.Ppack = dev_alloc<uint32_t>((size_t)ncs::tc_pack_words(pc.K, pc.Kstar, ncs::tc_block_cols(pc.K)));
    // on the context's stream: a device-wide synchronisation here would fail while another
    // host thread captures a CUDA graph (which a batch of contexts can do concurrently)
    CU(ncs::launch_tc_pack_b(T32d, pt, pc.K, d.Tpack, c->stream));
    CU(ncs::launch_tc_pack_b(P32d, pc.K, pc.Kstar, d.Ppack, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    dev_free(T32d);
    dev_free(P32d);
  }
  d.tc_err = dev_alloc<int>(1);
  CU(cudaMemset(d.tc_err, 0, sizeof(int)));
  d.TT64 = dev_upload(TT);
  d.TT32 = dev_upload(TT32);
  d.PT64 = dev_upload(PT);
  d.PT32 = dev_upload(PT32);
  d.zloc = dev_upload(pc.zloc);
  d.sloc = dev_upload(sl);
  d.I = dev_upload(pc.I);
  {
    // float-float log table: c_i = 1 + (i + 1/2)/64
    std::vector<float> lt(4 * 64);
    for (int i = 0; i < 64; ++i) {
      const double ci = 1.0 + (i + 0.5) / 64.0;
      const double L = std::log(ci), inv = 1.0 / ci;
      lt[4 * i + 0] = (float)L;
      lt[4 * i + 1] = (float)(L - (double)(float)L);
      lt[4 * i + 2] = (float)inv;
      lt[4 * i + 3] = (float)(inv - (double)(float)inv);
    }
    float* dl = dev_upload(lt);
    d.logtab = reinterpret_cast<float4*>(dl);
  }
  d.rep_p = dev_upload(rp);
  d.rep_off = dev_upload(ro);
  d.rep_rho = dev_upload(rr);
}

int finish(ncs_ctx* c, const Fail& f) {
  if (c) c->err = f.msg;
  if (c && log_level() > 0) std::fprintf(stderr, "ncs: %s\n", f.msg.c_str());
  return f.code;
}

// The device is bound at the first call that needs it; set-up (precompute, layout
// validation, tree construction) is host-only.
void ensure_device(ncs_ctx* c) {
  if (c->device_ready) {
    CU(cudaSetDevice(c->device));
    return;
  }
  CU(cudaGetDevice(&c->device));
  CU(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
  upload_operator(c);
  c->device_ready = true;
}

void ensure_layout(ncs_ctx* c) {
  if (!c->layout_dirty) return;
  DeviceData& d = c->d;
  const int64_t N = (int64_t)(c->centres.size() / 3);
  d.centres = dev_upload(c->centres);
  d.soff64 = dev_alloc<double>((size_t)N * d.p * 3);
  d.soff32 = dev_alloc<float>((size_t)N * d.p * 3);
  d.rho64 = dev_alloc<double>((size_t)N * d.p);
  d.rho32 = dev_alloc<float>((size_t)N * d.p);
  d.z = dev_alloc<double>((size_t)N * d.Kstar);
  if (c->prm.tensor_cores)  // TF32 hi/lo blocks of x or z for the tensor-core GEMMs
    d.Apack = dev_alloc<uint32_t>((size_t)ncs::tc_pack_words(N, std::max(d.K, d.Kstar), 128));
  d.N = N;
  CU(ncs::launch_skeleton_offsets(d, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  c->layout_dirty = false;
}

void check_ready(ncs_ctx* c) {
  if (!c) throw Fail{NCS_E_INPUT, "null context"};
  if (c->centres.empty()) throw Fail{NCS_E_STATE, "no patches: call ncs_set_patches first"};
  ensure_device(c);
  ensure_layout(c);
}

bool use_tree(const ncs_ctx* c) {
  if (c->method == NCS_METHOD_TREE) return true;
  if (c->method == NCS_METHOD_DIRECT) return false;
  return (int64_t)(c->centres.size() / 3) >= c->prm.tree_min_patches;
}

ncs::TreeOptions tree_options(const ncs_ctx* c, double grid_tol) {
  ncs::TreeOptions to;
  to.grid_tol = grid_tol;
  to.eps = c->pc.eps;
  to.item_patches = c->tune.item_patches;
  to.l2p_weight = c->tune.l2p_weight;
  return to;
}

// host part of the tree (Step 2 of Section 7)
void ensure_tree_host(ncs_ctx* c) {
  if (c->tree_built) return;
#ifdef _OPENMP
  // the thread count is an ICV of the calling host thread: the context's, on every build
  omp_set_num_threads(c->prm.threads > 0 ? c->prm.threads : omp_get_num_procs());
#endif
  ncs::tree_build(c->centres, c->pc, tree_options(c, c->prm.grid_tol), c->tree);
  c->tree_built = true;
}

void set_kernel_config(const ncs_ctx* c, ncs::TreeDevice& t) {
  t.cfg.p2l_tile = c->tune.p2l_tile;
  t.cfg.p2l_poly = c->tune.p2l_poly;
  t.cfg.direct_poly = c->tune.direct_poly;
  t.cfg.p2l_rsq = c->tune.p2l_rsq;
  t.cfg.direct_rsq = c->tune.direct_rsq;
}

// The mixed solve's inner FP32 products need only the accuracy of FP32 pair sums (~1e-6), so
// they may use incoming grids to a looser tolerance than the product's (fewer grid points
// and P2L pairs); the refinement residuals keep the product's tree. Below ~1e4 patches a
// tree product is bound by launch latency rather than by its pair sums, and a second tree
// would cost more set-up than it saves.
constexpr int64_t kInnerTreeMinPatches = 10000;
bool inner_tree_enabled(const ncs_ctx* c) {
  return c->prm.inner_grid_tol > c->prm.grid_tol && (int64_t)(c->centres.size() / 3) >= kInnerTreeMinPatches;
}

void ensure_inner_tree(ncs_ctx* c) {
  if (!inner_tree_enabled(c)) return;
  if (!c->tree_in_built) {
#ifdef _OPENMP
    omp_set_num_threads(c->prm.threads > 0 ? c->prm.threads : omp_get_num_procs());
#endif
    ncs::tree_build(c->centres, c->pc, tree_options(c, c->prm.inner_grid_tol), c->tree_in);
    c->tree_in_built = true;
  }
  if (!c->tree_in_uploaded) {
    ncs::tree_upload(c->tree_in, c->pc, c->tdev_in);
    c->tree_in_uploaded = true;
  }
  set_kernel_config(c, c->tdev_in);
}

// The product's tree; with the context's precision mixed, the inner tree as well (built
// with the product's, so that a solve finds both ready).
void ensure_tree(ncs_ctx* c) {
  ensure_tree_host(c);
  if (!c->tree_uploaded) {
    ncs::tree_upload(c->tree, c->pc, c->tdev);
    c->tree_uploaded = true;
  }
  set_kernel_config(c, c->tdev);
  if (c->precision == NCS_MIXED) ensure_inner_tree(c);
}

void outgoing(ncs_ctx* c, const double* x, int prec, cudaStream_t s) {
  if (prec == NCS_FP32 && c->prm.tensor_cores)
    CU(ncs::launch_tc_outgoing(c->d, x, c->d.tc_err, s));
  else
    CU(ncs::launch_outgoing(c->d, x, prec, s));
}

void apply_P(ncs_ctx* c, const double* x, double* y, int prec, cudaStream_t s) {
  if (prec == NCS_FP32 && c->prm.tensor_cores)
    CU(ncs::launch_tc_apply_P(c->d, x, y, c->d.tc_err, s));
  else
    CU(ncs::launch_apply_P(c->d, x, y, prec, s));
}

// A tensor-core kernel whose bounded wait gave up leaves the flag set (checked at
// synchronisation points).
void check_tc(ncs_ctx* c) {
  if (!c->prm.tensor_cores || !c->d.tc_err) return;
  int f = 0;
  CU(cudaMemcpy(&f, c->d.tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (f) {
    CU(cudaMemset(c->d.tc_err, 0, sizeof(int)));
    throw Fail{NCS_E_TIMEOUT, "tensor-core GEMM: bounded wait on its mbarrier gave up"};
  }
}

// z = field of x at the Zernike nodes (before P), on stream s.
void field(ncs_ctx* c, const double* x, int prec, cudaStream_t s) {
  outgoing(c, x, prec, s);
  if (use_tree(c)) {
    ensure_tree(c);
    const bool inner = c->inner_active && prec == NCS_FP32 && c->tree_in_uploaded;
    CU(ncs::launch_tree_field(c->d, inner ? c->tdev_in : c->tdev, c->pc.mode, prec, s));
  } else {
    CU(ncs::launch_direct_field(c->d, c->pc.mode, prec, c->pc.eps, s));
  }
}

void matvec(ncs_ctx* c, const double* x, double* y, int prec, cudaStream_t s) {
  field(c, x, prec, s);
  apply_P(c, x, y, prec, s);
}

double dev_dot(ncs_ctx* c, const double* a, const double* b, cudaStream_t s) {
  const int64_t n = c->d.N * c->d.K;
  CU(ncs::launch_dots(n, 1, a, n, b, c->partial, c->hdev, s));
  double h = 0.0;
  CU(cudaMemcpyAsync(&h, c->hdev, sizeof(double), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  return h;
}

void ensure_krylov(ncs_ctx* c, int maxit) {
  const int64_t n = c->d.N * c->d.K;
  if (c->Vcap < maxit + 1) {
    invalidate_graphs(c);
    dev_free(c->V);
    c->V = dev_alloc<double>((size_t)(maxit + 1) * n);
    c->Vcap = maxit + 1;
    dev_free(c->partial);
    dev_free(c->hdev);
    c->partial = dev_alloc<double>((size_t)ncs::kDotChunks * (maxit + 2));
    c->hdev = dev_alloc<double>(maxit + 2);
    // device GMRES state and arrays, one allocation
    dev_free(c->gmem);
    const size_t m1 = (size_t)maxit + 1, nb = (size_t)ncs::gmres_update_blocks(n);
    const size_t st_words = (sizeof(ncs::GmresState) + 7) / 8;
    const size_t words = st_words + m1 * maxit + 2 * (size_t)maxit + m1 + maxit + 2 * m1 + ncs::kDotChunks * m1 +
                         nb + (size_t)n;
    c->gmem = dev_alloc<double>(words);
    ncs::GmresDev& g = c->gd;
    double* q = c->gmem;
    g.maxit = maxit;
    g.st = reinterpret_cast<ncs::GmresState*>(q);
    q += st_words;
    g.H = q, q += m1 * maxit;
    g.cs = q, q += maxit;
    g.sn = q, q += maxit;
    g.g = q, q += m1;
    g.y = q, q += maxit;
    g.h1 = q, q += m1;
    g.h2 = q, q += m1;
    g.partial = q, q += ncs::kDotChunks * m1;
    g.pnorm = q, q += nb;
    g.vk = q;
  }
  if (!c->work) c->work = dev_alloc<double>(5 * (size_t)n);
  if (!c->st_host) CU(cudaHostAlloc((void**)&c->st_host, sizeof(ncs::GmresState), cudaHostAllocDefault));
}

// One Arnoldi step: w = A vk, two Gram-Schmidt passes, the Givens update, the next basis
// vector, and a copy of the device state into pinned host memory. Every argument is fixed
// for a given workspace and layout; the step's column index is read on the device.
void arnoldi_step(ncs_ctx* c, int prec, cudaStream_t s) {
  const int64_t n = c->d.N * c->d.K;
  double* w = c->work + 3 * n;
  matvec(c, c->gd.vk, w, prec, s);
  CU(ncs::launch_arnoldi_orthogonalize(n, c->V, w, c->gd, s));
  CU(cudaMemcpyAsync(c->st_host, c->gd.st, sizeof(ncs::GmresState), cudaMemcpyDeviceToHost, s));
}

// Captures arnoldi_step as a CUDA graph (once per precision and workspace). On any failure
// the context keeps launching the step directly (the same kernels) and says why.
void capture_step(ncs_ctx* c, int prec, int slot, cudaStream_t s) {
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    c->graphs_off = true;
    return;
  }
  const long long n0 = ncs::g_launches.load();
  bool ok = true;
  try {
    arnoldi_step(c, prec, s);
  } catch (const Fail& f) {
    ok = false;
    c->graph_note = f.msg;
  }
  const long long n1 = ncs::g_launches.load();
  ncs::g_launches.fetch_sub(n1 - n0);  // captured, not launched
  const cudaError_t e = cudaStreamEndCapture(s, &g);
  cudaGraphExec_t ge = nullptr;
  if (ok && e == cudaSuccess && g && cudaGraphInstantiate(&ge, g, 0) == cudaSuccess) {
    c->step_graph[slot] = ge;
    c->step_graph_kernels[slot] = n1 - n0;
  } else {
    cudaGetLastError();
    if (ok) c->graph_note = std::string("graph capture: ") + cudaGetErrorString(e);
    c->graphs_off = true;
  }
  if (g) cudaGraphDestroy(g);
}

// GMRES (x0 = 0, no restart) for A e = r with products at precision `prec`, its whole
// state on the device: CGS2 orthogonalisation, Givens rotations, residual estimate and
// back substitution in FP64 kernels. The host launches one step (a replay of the captured
// graph after the first) and reads the 48-byte state back. Returns the number of products;
// *est receives the estimated relative residual, e the iterate.
int gmres(ncs_ctx* c, const double* r, double* e, double tol, int prec, int maxit, double* est,
          cudaStream_t s) {
  const int64_t n = c->d.N * c->d.K;
  const double beta = std::sqrt(dev_dot(c, r, r, s));
  CU(cudaMemsetAsync(e, 0, n * sizeof(double), s));
  if (!std::isfinite(beta)) throw Fail{NCS_E_NUMERIC, "GMRES: non-finite right-hand side"};
  if (!(beta > 0.0)) {
    *est = 0.0;
    return 0;
  }
  ncs::GmresDev& gd = c->gd;
  maxit = std::min(maxit, gd.maxit);
  // the inner solves of a mixed solve run on their own tree: their own captured step
  const int slot = (c->inner_active && prec == NCS_FP32) ? 4 : prec;
  *c->st_host = ncs::GmresState{0, 0, ncs::kGmresRunning, maxit, beta, tol, 1.0, 0.0};
  CU(cudaMemcpyAsync(gd.st, c->st_host, sizeof(ncs::GmresState), cudaMemcpyHostToDevice, s));
  CU(ncs::launch_scale_copy(n, r, 1.0 / beta, c->V, s));
  CU(cudaMemcpyAsync(gd.vk, c->V, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  int steps = 0;
  while (steps < maxit) {
    if (steps > 0 && c->prm.cuda_graphs && !c->graphs_off && !c->step_graph[slot]) capture_step(c, prec, slot, s);
    if (steps > 0 && c->step_graph[slot]) {
      CU(cudaGraphLaunch(c->step_graph[slot], s));
      ncs::g_launches.fetch_add(c->step_graph_kernels[slot]);
      c->solve_stats[5] += 1.0;
    } else {
      arnoldi_step(c, prec, s);
    }
    CU(cudaStreamSynchronize(s));
    ++steps;
    const ncs::GmresState h = *c->st_host;
    if (log_level() > 1) std::fprintf(stderr, "ncs: gmres it %d est %.3e\n", h.m, h.res);
    if (h.done) break;
  }
  const ncs::GmresState h = *c->st_host;
  if (h.flag == ncs::kGmresNonFinite) throw Fail{NCS_E_NUMERIC, "GMRES: non-finite Arnoldi vector"};
  if (h.flag == ncs::kGmresBreakdown && h.m == 0) throw Fail{NCS_E_NUMERIC, "GMRES: breakdown (zero Hessenberg column)"};
  if (h.m > 0) {
    CU(ncs::launch_gmres_backsolve(gd, s));
    CU(ncs::launch_sub_combination(n, h.m, c->V, n, gd.y, e, 1.0, s));
  }
  CU(cudaStreamSynchronize(s));
  *est = h.flag == ncs::kGmresBreakdown ? 1.0 : h.res;
  c->solve_stats[0] += steps;
  return steps;
}

void validate_centres(int64_t N, const double* cen, double eps) {
  if (N < 1) throw Fail{NCS_E_INPUT, "N must be >= 1"};
  if (!cen) throw Fail{NCS_E_INPUT, "centres is NULL"};
  for (int64_t i = 0; i < N; ++i) {
    const double* c = cen + 3 * i;
    const double r2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    if (!std::isfinite(r2) || std::fabs(r2 - 1.0) > 2e-10)
      throw Fail{NCS_E_INPUT, "centre " + std::to_string(i) + " is not a unit vector"};
  }
  // geodesic separation >= 3 eps (Section 3), by a cell hash on chord distance
  const double chord_min = 2.0 * std::sin(1.5 * eps) * (1.0 - 1e-9);
  const double h = chord_min;
  std::unordered_map<uint64_t, std::vector<int64_t>> cells;
  cells.reserve((size_t)N * 2);
  auto key = [h](double x, double y, double z) {
    const int64_t a = (int64_t)std::floor(x / h) + (1 << 20), b = (int64_t)std::floor(y / h) + (1 << 20),
                  cc = (int64_t)std::floor(z / h) + (1 << 20);
    return ((uint64_t)a << 42) ^ ((uint64_t)b << 21) ^ (uint64_t)cc;
  };
  for (int64_t i = 0; i < N; ++i) cells[key(cen[3 * i], cen[3 * i + 1], cen[3 * i + 2])].push_back(i);
  // the first patch i (in index order) with a later patch j too close, and that j
  auto too_close = [&](int64_t i, int64_t* jout) {
    const double* c = cen + 3 * i;
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          auto it = cells.find(key(c[0] + dx * h, c[1] + dy * h, c[2] + dz * h));
          if (it == cells.end()) continue;
          for (int64_t j : it->second) {
            if (j <= i) continue;
            const double* e = cen + 3 * j;
            const double d2 = (c[0] - e[0]) * (c[0] - e[0]) + (c[1] - e[1]) * (c[1] - e[1]) +
                              (c[2] - e[2]) * (c[2] - e[2]);
            if (d2 < chord_min * chord_min) {
              if (jout) *jout = j;
              return true;
            }
          }
        }
    return false;
  };
  int64_t bad = N;
#pragma omp parallel for schedule(dynamic, 1024) reduction(min : bad)
  for (int64_t i = 0; i < N; ++i)
    if (i < bad && too_close(i, nullptr)) bad = i;
  if (bad < N) {
    int64_t j = -1;
    too_close(bad, &j);
    throw Fail{NCS_E_INPUT, "patches " + std::to_string(bad) + " and " + std::to_string(j) + " are closer than 3 eps"};
  }
}

ncs_ctx* new_ctx(const ncs_params* params) {
  ncs_ctx* c = new (std::nothrow) ncs_ctx();
  if (!c) throw Fail{NCS_E_OOM, "out of host memory"};
  if (params)
    c->prm = *params;
  else
    ncs_default_params(&c->prm);
  c->method = c->prm.method;
  return c;
}

void validate_params(const ncs_params& p) {
  if (p.npan < 2 || p.npan > 40 || p.nord < 2 || p.nord > 64) throw Fail{NCS_E_INPUT, "bad panel parameters"};
  if (!(p.id_tol > 0.0 && p.id_tol < 1e-2)) throw Fail{NCS_E_INPUT, "id_tol out of range"};
  if (!(p.id_ladder_max >= 0.0 && p.id_ladder_max <= 4.0)) throw Fail{NCS_E_INPUT, "id_ladder_max out of range"};
  if (!(p.grid_tol > 0.0 && p.grid_tol < 1e-1)) throw Fail{NCS_E_INPUT, "grid_tol out of range"};
  if (!(p.inner_grid_tol >= 0.0 && p.inner_grid_tol < 1e-1)) throw Fail{NCS_E_INPUT, "inner_grid_tol out of range"};
  if (p.gmres_maxit < 1 || p.gmres_maxit > 2000) throw Fail{NCS_E_INPUT, "gmres_maxit out of range"};
  if (p.method < 0 || p.method > 2) throw Fail{NCS_E_INPUT, "bad method"};
  if (p.mixed_residual != NCS_FP64 && p.mixed_residual != NCS_DF64)
    throw Fail{NCS_E_INPUT, "mixed_residual must be NCS_FP64 or NCS_DF64"};
}

bool tuning_valid(const ncs_tuning& t) {
  const auto poly_ok = [](int p) { return p == 0 || p == 2 || p == 4 || p == 6; };
  const auto rsq_ok = [](int r) { return r == 0 || r == 4 || r == 8; };
  return (t.p2l_tile == 8 || t.p2l_tile == 16) && poly_ok(t.p2l_poly) && poly_ok(t.direct_poly) &&
         rsq_ok(t.p2l_rsq) && rsq_ok(t.direct_rsq) && t.item_patches >= 8 && t.item_patches <= 64 &&
         t.item_patches % t.p2l_tile == 0 && t.l2p_weight >= 0.01 && t.l2p_weight <= 1.0;
}

// Applies a launch configuration; a change of the tree knobs drops the tree (rebuilt on
// the host, and uploaded, at the next product).
void apply_tuning(ncs_ctx* c, const ncs_tuning& t) {
  const bool rebuild = t.item_patches != c->tune.item_patches || t.l2p_weight != c->tune.l2p_weight;
  c->tune = t;
  invalidate_graphs(c);
  if (rebuild && (c->tree_built || c->tree_in_built)) drop_trees(c);
}

// Cache key of a workload: mode, K, eps, N (in half-octaves) and the shape of its tree
// (levels, per-mille of pair evaluations in the direct lists).
std::string tune_key(const ncs_ctx* c) {
  const ncs::TreeHost& t = c->tree;
  const int64_t N = (int64_t)(c->centres.size() / 3);
  const double share = (double)t.direct_pairs / std::max<double>(1.0, (double)(t.direct_pairs + t.p2l_pairs));
  char buf[160];
  std::snprintf(buf, sizeof buf, "m%d_K%d_e%.4g_N%d_L%d_d%d_g%.0e", c->pc.mode, c->pc.K, c->pc.eps,
                (int)std::lround(2.0 * std::log2((double)N)), t.levels, (int)std::lround(1000.0 * share),
                c->prm.grid_tol);
  return buf;
}

bool tune_cache_lookup(const char* path, const std::string& key, ncs_tuning* t) {
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[512], k[256];
  bool hit = false;
  ncs_tuning v{};
  while (std::fgets(line, sizeof line, f)) {
    if (std::sscanf(line, "ncs-tune-v2 %255s %d %d %d %d %lf %d %d", k, &v.p2l_tile, &v.p2l_poly, &v.direct_poly,
                    &v.item_patches, &v.l2p_weight, &v.p2l_rsq, &v.direct_rsq) == 8 &&
        key == k && tuning_valid(v)) {
      *t = v;
      hit = true;  // the last entry for a key wins
    }
  }
  std::fclose(f);
  return hit;
}

void tune_cache_store(const char* path, const std::string& key, const ncs_tuning& t) {
  FILE* f = std::fopen(path, "a");
  if (!f) throw Fail{NCS_E_INPUT, std::string("tune cache: cannot append to ") + path};
  std::fprintf(f, "ncs-tune-v2 %s %d %d %d %d %.17g %d %d\n", key.c_str(), t.p2l_tile, t.p2l_poly, t.direct_poly,
               t.item_patches, t.l2p_weight, t.p2l_rsq, t.direct_rsq);
  std::fclose(f);
}

// Far-field extent of the ID ladder for one sphere of a batch, from its patch count: every
// extra representation costs one sketch CPQR and T assembly in the precompute (~10 ms of FP64
// device work each at K = 128) and saves pair evaluations in every product. Measured on GB300
// (K = 128, mixed solve to 1e-8, precompute + solve seconds for ladder extents 0 / 0.1 / 1.0):
// N = 200: 0.16 / 0.24 / 0.30; N = 700: 0.24 / 0.27 / 0.32; N = 2000: 0.46 / 0.35 / 0.37;
// N = 5000: 1.14 / 0.53 / 0.52. Hence no ladder below 1000 patches, a short one below 3000.
double batch_ladder_extent(int64_t N) {
  if (N < 1000) return 0.0;
  if (N < 3000) return 0.1;
  return 1.0;
}

// ---- grouped solve of small spheres (ncs_batch_solve). Spheres with few patches keep
// only a few hundred blocks busy per product and spend most of a solve in launch latency;
// a group of them (common K and mode) is solved as one concatenated system whose products,
// Krylov steps and refinement sweeps each take one launch per stage for all instances.

struct GroupResult {
  double scalar = 0.0, Is = 0.0, rel = 1.0;
  int iters = 0;
  int status = NCS_OK;
};

// Device buffers of one group, freed together.
struct GroupStore {
  std::vector<void*> ptrs;
  template <typename T>
  T* up(const std::vector<T>& h) {
    T* p = dev_upload(h);
    ptrs.push_back(p);
    return p;
  }
  template <typename T>
  T* alloc(size_t n) {
    T* p = dev_alloc<T>(n);
    ptrs.push_back(p);
    return p;
  }
  ~GroupStore() {
    for (void* p : ptrs) cudaFree(p);
  }
};

// Patch frame of unit centre c on the host (the frame of the device kernels).
void host_frame(const double* c, double* e1, double* e2) {
  e1[0] = -c[1];
  e1[1] = c[0];
  e1[2] = 0.0;
  const double na2 = e1[0] * e1[0] + e1[1] * e1[1];
  if (na2 >= 1e-24) {
    const double inv = 1.0 / std::sqrt(na2);
    e1[0] *= inv;
    e1[1] *= inv;
  } else {
    e1[0] = 1.0;
    e1[1] = 0.0;
  }
  e2[0] = c[1] * e1[2] - c[2] * e1[1];
  e2[1] = c[2] * e1[0] - c[0] * e1[2];
  e2[2] = c[0] * e1[1] - c[1] * e1[0];
}

// Solves the instances cs (same K and mode, direct products) by the mixed scheme of
// ncs_solve: FP32 inner GMRES for every instance still refining, in lock step, then the
// residual b - A x recomputed at prm.mixed_residual precision; an instance leaves the
// sweep once its residual meets tol or stops decreasing. With `graphs` the Krylov step
// (product, Arnoldi kernels, copy of the states) is captured once as a CUDA graph and
// replayed; the caller guarantees that no other host thread uses the device meanwhile.
// Per-instance results in res.
void group_solve(const std::vector<ncs_ctx*>& cs, double tol, bool graphs, cudaStream_t s, std::vector<GroupResult>& res) {
  const int B = (int)cs.size();
  const ncs::Precomputed& pc0 = cs[0]->pc;
  const int K = pc0.K, Kstar = pc0.Kstar, mode = pc0.mode;
  const ncs_params& prm = cs[0]->prm;
  const int maxit = prm.gmres_maxit;
  res.assign(B, GroupResult{});
  // host tables
  std::vector<int64_t> pbase(B + 1, 0), tt_off(B), roff;
  std::vector<int> pinst, ptot(B), nrep(B), repbase(B), rep_p, rep_off;
  std::vector<double> rep_rho, ieps(B), zloc, I, centres;
  std::vector<double> TT;
  int pmax = 1;
  int64_t maxseg = 1;
  for (int b = 0; b < B; ++b) {
    const ncs_ctx* c = cs[b];
    const ncs::Precomputed& pc = c->pc;
    if (pc.K != K || pc.Kstar != Kstar || pc.mode != mode) throw Fail{NCS_E_INPUT, "group: mixed K or mode"};
    const int64_t N = (int64_t)(c->centres.size() / 3);
    pbase[b + 1] = pbase[b] + N;
    maxseg = std::max<int64_t>(maxseg, N * K);
    ieps[b] = pc.eps;
    nrep[b] = (int)pc.reps.size();
    repbase[b] = (int)rep_p.size();
    int pt = 0;
    for (const auto& r : pc.reps) {
      rep_p.push_back(r.p);
      rep_off.push_back(pt);
      rep_rho.push_back(r.rho_min);
      pt += r.p;
      pmax = std::max(pmax, r.p);
    }
    ptot[b] = pt;
    tt_off[b] = (int64_t)TT.size();
    TT.resize(TT.size() + (size_t)K * pt);
    double* Tb = TT.data() + tt_off[b];
    for (const auto& r : pc.reps) {
      const int o = rep_off[repbase[b] + (int)(&r - pc.reps.data())];
      for (int m = 0; m < r.p; ++m)
        for (int k = 0; k < K; ++k) Tb[(size_t)k * pt + o + m] = r.T[(size_t)m * K + k];
    }
    zloc.insert(zloc.end(), pc.zloc.begin(), pc.zloc.end());
    I.insert(I.end(), pc.I.begin(), pc.I.end());
    centres.insert(centres.end(), c->centres.begin(), c->centres.end());
    for (int64_t i = 0; i < N; ++i) pinst.push_back(b);
  }
  const int64_t P = pbase[B];
  const int64_t n = P * K;
  // coefficient offsets and skeleton offsets (global frame) of every patch
  roff.resize(P);
  int64_t R = 0;
  for (int64_t i = 0; i < P; ++i) {
    roff[i] = R;
    R += ptot[pinst[i]];
  }
  std::vector<double> soff(3 * (size_t)R);
  for (int64_t i = 0; i < P; ++i) {
    const ncs::Precomputed& pc = cs[pinst[i]]->pc;
    const double* c = &centres[3 * i];
    double e1[3], e2[3];
    host_frame(c, e1, e2);
    int64_t q = roff[i];
    for (const auto& r : pc.reps)
      for (int m = 0; m < r.p; ++m, ++q) {
        const double* o = &r.sloc[3 * (size_t)m];
        for (int a = 0; a < 3; ++a) soff[3 * q + a] = o[0] * e1[a] + o[1] * e2[a] + o[2] * c[a];
      }
  }
  std::vector<double> PT((size_t)Kstar * K);
  for (int j = 0; j < K; ++j)
    for (int q = 0; q < Kstar; ++q) PT[(size_t)q * K + j] = pc0.P[(size_t)j * Kstar + q];
  std::vector<float> lt(4 * 64);
  for (int i = 0; i < 64; ++i) {
    const double ci = 1.0 + (i + 0.5) / 64.0;
    const double L = std::log(ci), inv = 1.0 / ci;
    lt[4 * i + 0] = (float)L;
    lt[4 * i + 1] = (float)(L - (double)(float)L);
    lt[4 * i + 2] = (float)inv;
    lt[4 * i + 3] = (float)(inv - (double)(float)inv);
  }
  GroupStore st;
  ncs::GroupDev g;
  g.B = B;
  g.K = K;
  g.Kstar = Kstar;
  g.mode = mode;
  g.maxit = maxit;
  g.pmax = pmax;
  g.seg_blocks = ncs::group_seg_blocks(maxseg);
  g.P = P;
  g.pinst = st.up(pinst);
  g.pbase = st.up(pbase);
  g.roff = st.up(roff);
  g.inst_ptot = st.up(ptot);
  g.tt_off = st.up(tt_off);
  g.inst_eps = st.up(ieps);
  g.inst_nrep = st.up(nrep);
  g.inst_repbase = st.up(repbase);
  g.rep_p = st.up(rep_p);
  g.rep_off = st.up(rep_off);
  g.rep_rho = st.up(rep_rho);
  g.zloc = st.up(zloc);
  g.centres = st.up(centres);
  g.soff64 = st.up(soff);
  g.soff32 = st.up(std::vector<float>(soff.begin(), soff.end()));
  g.rho64 = st.alloc<double>(R);
  g.rho32 = st.alloc<float>(R);
  g.TT64 = st.up(TT);
  g.TT32 = st.up(std::vector<float>(TT.begin(), TT.end()));
  g.z = st.alloc<double>((size_t)P * Kstar);
  g.I = st.up(I);
  g.logtab = reinterpret_cast<const float4*>(st.up(lt));
  const size_t m1 = (size_t)maxit + 1;
  g.st = reinterpret_cast<ncs::GmresState*>(st.alloc<double>(B * ((sizeof(ncs::GmresState) + 7) / 8)));
  g.H = st.alloc<double>(B * m1 * maxit);
  g.cs = st.alloc<double>((size_t)B * maxit);
  g.sn = st.alloc<double>((size_t)B * maxit);
  g.g = st.alloc<double>(B * m1);
  g.y = st.alloc<double>((size_t)B * maxit);
  g.h1 = st.alloc<double>(B * m1);
  g.h2 = st.alloc<double>(B * m1);
  g.pnorm = st.alloc<double>((size_t)B * g.seg_blocks);
  g.vk = st.alloc<double>(n);
  // the Zernike transform y = x + P z of ncs_solve's product (P is common to the group)
  DeviceData dd;
  dd.N = P;
  dd.K = K;
  dd.Kstar = Kstar;
  dd.z = g.z;
  dd.PT64 = st.up(PT);
  dd.PT32 = st.up(std::vector<float>(PT.begin(), PT.end()));
  double* V = st.alloc<double>(m1 * n);
  double* work = st.alloc<double>(5 * (size_t)n);
  double *bv = work, *x = work + n, *r = work + 2 * n, *corr = work + 3 * n, *w = work + 4 * n;
  double* dsc = st.alloc<double>(B);  // per-instance scalars (dots, scale factors)
  ncs::GmresState* sth = nullptr;
  CU(cudaHostAlloc((void**)&sth, B * sizeof(ncs::GmresState), cudaHostAllocDefault));
  std::unique_ptr<ncs::GmresState, decltype(&cudaFreeHost)> sth_guard(sth, &cudaFreeHost);
  std::vector<double> hb(B);
  auto seg_dots = [&](const double* a, const double* c2) {
    CU(ncs::launch_group_dots(g, a, c2, dsc, s));
    CU(cudaMemcpyAsync(hb.data(), dsc, B * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return hb;
  };
  auto product = [&](const double* in, double* out, int prec) {
    CU(ncs::launch_group_field(g, in, prec, s));
    CU(ncs::launch_apply_P(dd, in, out, prec, s));
  };
  // right-hand side b_i = P 1 (eq. opinteqnsdisc)
  {
    std::vector<double> P1(K, 0.0);
    for (int j = 0; j < K; ++j)
      for (int q = 0; q < Kstar; ++q) P1[j] += pc0.P[(size_t)j * Kstar + q];
    std::vector<double> bh((size_t)n);
    for (int64_t i = 0; i < P; ++i) std::memcpy(&bh[(size_t)i * K], P1.data(), K * sizeof(double));
    CU(cudaMemcpyAsync(bv, bh.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  std::vector<double> bnorm = seg_dots(bv, bv);
  for (double& v : bnorm) v = std::sqrt(v);
  CU(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  CU(cudaMemcpyAsync(r, bv, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  std::vector<char> active(B, 1);
  // one Krylov step of every running instance: w = A vk, orthogonalisation, Givens, the
  // next basis vector, and the states copied into pinned host memory
  auto krylov_step = [&]() {
    product(g.vk, w, NCS_FP32);
    CU(ncs::launch_group_arnoldi(g, V, w, s));
    CU(cudaMemcpyAsync(sth, g.st, B * sizeof(ncs::GmresState), cudaMemcpyDeviceToHost, s));
  };
  std::unique_ptr<std::remove_pointer<cudaGraphExec_t>::type, decltype(&cudaGraphExecDestroy)> graph(
      nullptr, &cudaGraphExecDestroy);
  long long graph_kernels = 0;
  auto capture = [&]() {
    graphs = false;  // one attempt; on failure the step keeps launching directly
    cudaGraph_t gr = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    const long long n0 = ncs::g_launches.load();
    bool ok = true;
    try {
      krylov_step();
    } catch (const Fail&) {
      ok = false;
    }
    const long long n1 = ncs::g_launches.load();
    ncs::g_launches.fetch_sub(n1 - n0);  // captured, not launched
    const cudaError_t e = cudaStreamEndCapture(s, &gr);
    cudaGraphExec_t ge = nullptr;
    if (ok && e == cudaSuccess && gr && cudaGraphInstantiate(&ge, gr, 0) == cudaSuccess) {
      graph.reset(ge);
      graph_kernels = n1 - n0;
    } else {
      cudaGetLastError();
    }
    if (gr) cudaGraphDestroy(gr);
  };
  // inner FP32 GMRES (x0 = 0, no restart) of every active instance for A corr = r
  auto inner = [&]() {
    std::vector<double> beta = seg_dots(r, r);
    std::vector<double> scale(B, 0.0);
    for (int b = 0; b < B; ++b) {
      beta[b] = std::sqrt(beta[b]);
      const bool run = active[b] && std::isfinite(beta[b]) && beta[b] > 0.0;
      const double itol = std::min(std::max(0.3 * tol / res[b].rel, 3e-6), 0.5);
      sth[b] = ncs::GmresState{0, run ? 0 : 1, run ? ncs::kGmresRunning : ncs::kGmresConverged, maxit,
                               run ? beta[b] : 1.0, itol, run ? 1.0 : 0.0, 0.0};
      scale[b] = run ? 1.0 / beta[b] : 0.0;
      if (active[b] && !std::isfinite(beta[b])) {
        res[b].status = NCS_E_NUMERIC;
        active[b] = 0;
      }
    }
    CU(cudaMemcpyAsync(g.st, sth, B * sizeof(ncs::GmresState), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(dsc, scale.data(), B * sizeof(double), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(V, r, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CU(ncs::launch_group_scale(g, dsc, V, s));
    CU(cudaMemcpyAsync(g.vk, V, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CU(cudaStreamSynchronize(s));
    for (int step = 0; step < maxit; ++step) {
      std::vector<char> running(B);
      bool any = false;
      for (int b = 0; b < B; ++b) any |= (running[b] = !sth[b].done);
      if (!any) break;
      if (step > 0 && graphs && !graph) capture();
      if (step > 0 && graph) {
        CU(cudaGraphLaunch(graph.get(), s));
        ncs::g_launches.fetch_add(graph_kernels);
      } else {
        krylov_step();
      }
      CU(cudaStreamSynchronize(s));
      for (int b = 0; b < B; ++b) res[b].iters += running[b];
    }
    for (int b = 0; b < B; ++b)
      if (active[b] && (sth[b].flag == ncs::kGmresNonFinite || (sth[b].flag == ncs::kGmresBreakdown && sth[b].m == 0))) {
        res[b].status = NCS_E_NUMERIC;
        active[b] = 0;
      }
    CU(ncs::launch_group_solution(g, V, corr, s));
  };
  for (int outer = 0; outer < 20; ++outer) {
    bool any = false;
    for (int b = 0; b < B; ++b) {
      if (active[b] && res[b].rel <= tol) active[b] = 0;
      any |= (bool)active[b];
    }
    if (!any) break;
    inner();
    // instances that ran no step (inactive) have corr = 0 on their segment
    CU(ncs::launch_axpby(n, 1.0, corr, 1.0, x, s));
    product(x, r, prm.mixed_residual);
    CU(ncs::launch_axpby(n, 1.0, bv, -1.0, r, s));
    const std::vector<double> rr = seg_dots(r, r);
    for (int b = 0; b < B; ++b) {
      if (!active[b]) continue;
      ++res[b].iters;
      const double newrel = std::sqrt(rr[b]) / bnorm[b];
      if (!std::isfinite(newrel)) {
        res[b].status = NCS_E_NUMERIC;
        active[b] = 0;
        continue;
      }
      const bool stalled = newrel > 0.9 * res[b].rel && outer > 0;
      res[b].rel = newrel;
      if (stalled) active[b] = 0;
    }
    if (log_level() > 0) {
      int left = 0;
      for (int b = 0; b < B; ++b) left += active[b];
      std::fprintf(stderr, "ncs: group refinement %d: %d of %d instances still refining\n", outer, left, B);
    }
  }
  // I_sigma = I . sum_i f_i (eq. getI), then mu or C
  CU(ncs::launch_group_isigma(g, x, dsc, s));
  CU(cudaMemcpyAsync(hb.data(), dsc, B * sizeof(double), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  for (int b = 0; b < B; ++b) {
    GroupResult& o = res[b];
    o.Is = hb[b];
    o.scalar = mode == NCS_INTERIOR ? 1.0 / (3.0 * o.Is) - 0.6 : 4.0 * M_PI * o.Is;
    if (o.status == NCS_OK && !(o.rel <= tol)) o.status = NCS_E_NOCONV;
  }
}

}  // namespace

extern "C" {

void ncs_default_params(ncs_params* p) {
  if (!p) return;
  p->npan = 13;
  p->nord = 20;
  p->ntheta_fine = 0;
  p->id_tol = 1e-11;
  p->threads = 0;
  p->grid_tol = 1e-8;
  p->method = NCS_METHOD_AUTO;
  p->tree_min_patches = 128;
  p->gmres_maxit = 200;
  p->verbose = 0;
  p->mixed_residual = NCS_DF64;
  p->tensor_cores = 1;
  p->residual_update = 1;
  p->id_ladder_max = 1.0;
  p->device_precompute = 1;
  p->cuda_graphs = 1;
  p->batch_ladder_by_n = 1;
  p->batch_grouped = 1;
  p->inner_grid_tol = 1e-5;
}

int ncs_create(double eps, int mode, int K, const ncs_params* params, ncs_ctx** out) {
  if (!out) return NCS_E_INPUT;
  *out = nullptr;
  ncs_ctx* c = nullptr;
  try {
    if (!(eps > 0.0 && eps < 1.0)) throw Fail{NCS_E_INPUT, "eps must be in (0, 1)"};
    if (mode != NCS_EXTERIOR && mode != NCS_INTERIOR) throw Fail{NCS_E_INPUT, "mode must be 0 or 1"};
    if (K < 1 || K > 2000) throw Fail{NCS_E_INPUT, "K must be in [1, 2000]"};
    c = new_ctx(params);
    validate_params(c->prm);
    ncs::PrecomputeOptions o;
    o.npan = c->prm.npan;
    o.nord = c->prm.nord;
    o.ntheta_fine = c->prm.ntheta_fine;
    o.id_tol = c->prm.id_tol;
    o.threads = c->prm.threads;
    o.id_ladder_max = c->prm.id_ladder_max;
    o.device_sketch = c->prm.device_precompute != 0;
    o.device_colloc = c->prm.device_precompute != 0;
    try {
      ncs::precompute(eps, mode, K, o, c->pc);
    } catch (const std::exception& e) {
      throw Fail{NCS_E_NUMERIC, std::string("precompute: ") + e.what()};
    }
    if (log_level() > 0)
      std::fprintf(stderr, "ncs: precompute eps=%g K=%d p=%d nf=%d (%.2fs + %.2fs)\n", eps, K, c->pc.p, c->pc.nf,
                   c->pc.seconds_onepatch, c->pc.seconds_id);
    *out = c;
    return NCS_OK;
  } catch (const Fail& f) {
    if (c) {
      free_all(c);
      delete c;
    }
    if (log_level() > 0) std::fprintf(stderr, "ncs_create: %s\n", f.msg.c_str());
    return f.code;
  } catch (const std::bad_alloc&) {
    if (c) {
      free_all(c);
      delete c;
    }
    return NCS_E_OOM;
  }
}

int ncs_create_from_operators(double eps, int mode, int K, int nrep, const double* rho_min, const int* p,
                              const double* T, const double* skel_t, const double* skel_theta, const double* I,
                              const ncs_params* params, ncs_ctx** out) {
  if (!out) return NCS_E_INPUT;
  *out = nullptr;
  ncs_ctx* c = nullptr;
  try {
    if (!(eps > 0.0 && eps < 1.0)) throw Fail{NCS_E_INPUT, "eps must be in (0, 1)"};
    if (mode != NCS_EXTERIOR && mode != NCS_INTERIOR) throw Fail{NCS_E_INPUT, "mode must be 0 or 1"};
    if (K < 1 || K > 2000 || nrep < 1 || nrep > 64) throw Fail{NCS_E_INPUT, "K or nrep out of range"};
    if (!rho_min || !p || !T || !skel_t || !skel_theta || !I) throw Fail{NCS_E_INPUT, "NULL operator array"};
    c = new_ctx(params);
    validate_params(c->prm);
    c->from_operator = true;
    ncs::precompute_zernike(eps, K, c->pc);
    c->pc.mode = mode;
    c->pc.I.assign(I, I + K);
    size_t off = 0;
    for (int r = 0; r < nrep; ++r) {
      if (p[r] < 1 || p[r] > 100000) throw Fail{NCS_E_INPUT, "p out of range"};
      if (!(rho_min[r] >= 2.0 * eps * (1.0 - 1e-12)) || (r > 0 && !(rho_min[r] > rho_min[r - 1])))
        throw Fail{NCS_E_INPUT, "far-field radii must start at >= 2 eps and increase"};
      ncs::OutRep rep;
      rep.rho_min = rho_min[r];
      rep.p = p[r];
      rep.T.assign(T + off * K, T + (off + p[r]) * K);
      rep.st.assign(skel_t + off, skel_t + off + p[r]);
      rep.sth.assign(skel_theta + off, skel_theta + off + p[r]);
      rep.sloc.resize(3 * (size_t)p[r]);
      for (int m = 0; m < p[r]; ++m) {
        if (!(rep.st[m] >= 0.0 && rep.st[m] <= eps)) throw Fail{NCS_E_INPUT, "skeleton t outside [0, eps]"};
        ncs::local_offset(rep.st[m], rep.sth[m], &rep.sloc[3 * (size_t)m]);
      }
      for (double v : rep.T)
        if (!std::isfinite(v)) throw Fail{NCS_E_INPUT, "non-finite T"};
      c->pc.reps.push_back(std::move(rep));
      off += p[r];
    }
    c->pc.p = c->pc.reps[0].p;
    c->pc.T = c->pc.reps[0].T;
    c->pc.st = c->pc.reps[0].st;
    c->pc.sth = c->pc.reps[0].sth;
    c->pc.sloc = c->pc.reps[0].sloc;
    *out = c;
    return NCS_OK;
  } catch (const Fail& f) {
    if (c) {
      free_all(c);
      delete c;
    }
    return f.code;
  } catch (const std::bad_alloc&) {
    if (c) {
      free_all(c);
      delete c;
    }
    return NCS_E_OOM;
  }
}

int ncs_create_from_operator(double eps, int mode, int K, int p, const double* T, const double* skel_t,
                             const double* skel_theta, const double* I, const ncs_params* params, ncs_ctx** out) {
  const double rho = 2.0 * eps;
  return ncs_create_from_operators(eps, mode, K, 1, &rho, &p, T, skel_t, skel_theta, I, params, out);
}

int ncs_get_reps(const ncs_ctx* c, int* nrep, double* rho_min, int* p) {
  if (!c || !nrep) return NCS_E_INPUT;
  const int n = (int)c->pc.reps.size();
  if (rho_min && p) {
    if (*nrep < n) return NCS_E_INPUT;
    for (int r = 0; r < n; ++r) {
      rho_min[r] = c->pc.reps[r].rho_min;
      p[r] = c->pc.reps[r].p;
    }
  }
  *nrep = n;
  return NCS_OK;
}

int ncs_set_precision(ncs_ctx* c, int precision) {
  if (!c) return NCS_E_INPUT;
  if (precision != NCS_FP64 && precision != NCS_FP32 && precision != NCS_MIXED && precision != NCS_DF64) {
    c->err = "ncs_set_precision: bad precision";
    return NCS_E_INPUT;
  }
  c->precision = precision;
  return NCS_OK;
}

int ncs_get_rep(const ncs_ctx* c, int r, double* T, double* skel_t, double* skel_theta) {
  if (!c || r < 0 || r >= (int)c->pc.reps.size()) return NCS_E_INPUT;
  const ncs::OutRep& rep = c->pc.reps[r];
  if (T) std::memcpy(T, rep.T.data(), rep.T.size() * sizeof(double));
  if (skel_t) std::memcpy(skel_t, rep.st.data(), rep.st.size() * sizeof(double));
  if (skel_theta) std::memcpy(skel_theta, rep.sth.data(), rep.sth.size() * sizeof(double));
  return NCS_OK;
}

int ncs_info(const ncs_ctx* c, int64_t* out, int n) {
  if (!c || !out) return NCS_E_INPUT;
  const int64_t v[13] = {c->pc.K,
                         c->pc.Kstar,
                         c->pc.p,
                         c->pc.M,
                         c->pc.nf,
                         (int64_t)(c->centres.size() / 3),
                         c->pc.nrad,
                         c->tree_built ? (int64_t)c->tree.levels : 0,
                         c->tree_built ? c->tree.total_grid_points : 0,
                         c->tree_built ? c->tree.pairs_per_matvec : 0,
                         (int64_t)(c->centres.size() / 3) * ((int64_t)(c->centres.size() / 3) - 1) *
                             (int64_t)c->pc.p * c->pc.Kstar,
                         c->tree_in_built ? c->tree_in.total_grid_points : 0,
                         c->tree_in_built ? c->tree_in.pairs_per_matvec : 0};
  for (int i = 0; i < n && i < 13; ++i) out[i] = v[i];
  return NCS_OK;
}

int ncs_timings(const ncs_ctx* c, double* out, int n) {
  if (!c || !out) return NCS_E_INPUT;
  if (n > 0) out[0] = c->pc.seconds_onepatch;
  if (n > 1) out[1] = c->pc.seconds_id;
  if (n > 2) out[2] = c->pc.sketch_on_device ? 1.0 : 0.0;
  if (n > 3) out[3] = c->pc.seconds_sketch;
  if (n > 4) out[4] = c->pc.seconds_cpqr;
  if (n > 5) out[5] = c->pc.seconds_assemble;
  if (n > 6) out[6] = c->pc.colloc_on_device ? 1.0 : 0.0;
  if (n > 7) out[7] = c->pc.seconds_colloc;
  if (n > 8) out[8] = c->pc.seconds_lu;
  return NCS_OK;
}

int ncs_get_operator(const ncs_ctx* c, double* T, double* skel_t, double* skel_theta, double* I, double* P,
                     double* zr, double* zth) {
  if (!c) return NCS_E_INPUT;
  const ncs::Precomputed& pc = c->pc;
  if (T) std::memcpy(T, pc.T.data(), pc.T.size() * sizeof(double));
  if (skel_t) std::memcpy(skel_t, pc.st.data(), pc.st.size() * sizeof(double));
  if (skel_theta) std::memcpy(skel_theta, pc.sth.data(), pc.sth.size() * sizeof(double));
  if (I) std::memcpy(I, pc.I.data(), pc.I.size() * sizeof(double));
  if (P) std::memcpy(P, pc.P.data(), pc.P.size() * sizeof(double));
  if (zr) std::memcpy(zr, pc.zr.data(), pc.zr.size() * sizeof(double));
  if (zth) std::memcpy(zth, pc.zth.data(), pc.zth.size() * sizeof(double));
  return NCS_OK;
}

int ncs_get_onepatch(const ncs_ctx* c, double* trad, double* beta) {
  if (!c) return NCS_E_INPUT;
  if (c->from_operator) return NCS_E_STATE;
  if (trad) std::memcpy(trad, c->pc.trad.data(), c->pc.trad.size() * sizeof(double));
  if (beta) std::memcpy(beta, c->pc.beta.data(), c->pc.beta.size() * sizeof(double));
  return NCS_OK;
}

int ncs_set_patches(ncs_ctx* c, int64_t N, const double* centres) {
  if (!c) return NCS_E_INPUT;
  try {
    validate_centres(N, centres, c->pc.eps);
    if (c->device_ready) CU(cudaSetDevice(c->device));
    free_layout(c);
    c->centres.assign(centres, centres + 3 * N);
    c->layout_dirty = true;
    if (use_tree(c)) ensure_tree_host(c);
    return NCS_OK;
  } catch (const Fail& f) {
    return finish(c, f);
  } catch (const std::bad_alloc&) {
    return finish(c, Fail{NCS_E_OOM, "out of host memory"});
  } catch (const std::exception& e) {
    return finish(c, Fail{NCS_E_INPUT, std::string("set_patches: ") + e.what()});
  }
}

int ncs_tree_pairs(ncs_ctx* c, int64_t* count, int* target, int* source, int* level, int* kind) {
  if (!c || !count) return NCS_E_INPUT;
  try {
    if (c->centres.empty()) throw Fail{NCS_E_STATE, "no patches: call ncs_set_patches first"};
    std::vector<int> t, s, l, k;
    ncs::tree_pairs(c->centres, c->pc, tree_options(c, c->prm.grid_tol), t, s, l, k);
    if (target && source && level && kind) {
      if (*count < (int64_t)t.size()) throw Fail{NCS_E_INPUT, "pair buffers too small"};
      std::memcpy(target, t.data(), t.size() * sizeof(int));
      std::memcpy(source, s.data(), s.size() * sizeof(int));
      std::memcpy(level, l.data(), l.size() * sizeof(int));
      std::memcpy(kind, k.data(), k.size() * sizeof(int));
    }
    *count = (int64_t)t.size();
    return NCS_OK;
  } catch (const Fail& f) {
    return finish(c, f);
  } catch (const std::exception& e) {
    return finish(c, Fail{NCS_E_INPUT, std::string("tree: ") + e.what()});
  }
}

int ncs_tree_stats(ncs_ctx* c, int64_t* out, int n) {
  if (!c || !out) return NCS_E_INPUT;
  try {
    if (c->centres.empty()) throw Fail{NCS_E_STATE, "no patches: call ncs_set_patches first"};
    ensure_tree_host(c);
    const ncs::TreeHost& t = c->tree;
    const int64_t v[11] = {t.levels, (int64_t)t.gR.size(), t.total_grid_points, (int64_t)t.witem_group.size(),
                           t.p2l_pairs, t.direct_pairs, t.l2p_evals, t.pd_off.empty() ? 0 : t.pd_off.back(),
                           (int64_t)t.shapes.size(), (int64_t)t.l2l_child.size(), t.l2l_evals};
    for (int i = 0; i < n && i < 11; ++i) out[i] = v[i];
    return NCS_OK;
  } catch (const Fail& f) {
    return finish(c, f);
  } catch (const std::exception& e) {
    return finish(c, Fail{NCS_E_INPUT, std::string("tree: ") + e.what()});
  }
}

int ncs_set_method(ncs_ctx* c, int method) {
  if (!c) return NCS_E_INPUT;
  if (method < 0 || method > 2) return finish(c, Fail{NCS_E_INPUT, "bad method"});
  if (method != c->method) invalidate_graphs(c);
  c->method = method;
  if (!c->centres.empty() && use_tree(c)) {
    try {
      ensure_tree_host(c);
    } catch (const Fail& f) {
      return finish(c, f);
    } catch (const std::exception& e) {
      return finish(c, Fail{NCS_E_INPUT, std::string("tree: ") + e.what()});
    }
  }
  return NCS_OK;
}

int ncs_matvec_dev(ncs_ctx* c, const double* x, double* y, int precision, void* stream) {
  if (c && precision == NCS_PRECISION_DEFAULT) precision = c->precision == NCS_MIXED ? NCS_FP32 : c->precision;
  try {
    if (!c) throw Fail{NCS_E_INPUT, "null context"};
    if (!x || !y) throw Fail{NCS_E_INPUT, "NULL vector"};
    if (precision != NCS_FP64 && precision != NCS_FP32 && precision != NCS_DF64)
      throw Fail{NCS_E_INPUT, "precision must be FP64, DF64 or FP32"};
    check_ready(c);
    matvec(c, x, y, precision, (cudaStream_t)stream);
    return NCS_OK;
  } catch (const Fail& f) {
    return finish(c, f);
  } catch (const std::exception& e) {
    return finish(c, Fail{NCS_E_INPUT, e.what()});
  }
}

int ncs_field_dev(ncs_ctx* c, const double* x, double* z, int precision, void* stream) {
  if (c && precision == NCS_PRECISION_DEFAULT) precision = c->precision == NCS_MIXED ? NCS_FP32 : c->precision;
  try {
    if (!c) throw Fail{NCS_E_INPUT, "null context"};
    if (!x || !z) throw Fail{NCS_E_INPUT, "NULL vector"};
    if (precision != NCS_FP64 && precision != NCS_FP32 && precision != NCS_DF64)
      throw Fail{NCS_E_INPUT, "precision must be FP64, DF64 or FP32"};
    check_ready(c);
    cudaStream_t s = (cudaStream_t)stream;
    field(c, x, precision, s);
    CU(cudaMemcpyAsync(z, c->d.z, (size_t)c->d.N * c->d.Kstar * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return NCS_OK;
  } catch (const Fail& f) {
    return finish(c, f);
  } catch (const std::exception& e) {
    return finish(c, Fail{NCS_E_INPUT, e.what()});
  }
}

int ncs_profile_matvec(ncs_ctx* c, const double* x, double* y, int precision, void* stream, double* ms, int n) {
  if (c && precision == NCS_PRECISION_DEFAULT) precision = c->precision == NCS_MIXED ? NCS_FP32 : c->precision;
  cudaEvent_t ev[8] = {};
  int rc = NCS_OK;
  try {
    if (!c) throw Fail{NCS_E_INPUT, "null context"};
    if (!x || !y || !ms) throw Fail{NCS_E_INPUT, "NULL argument"};
    if (precision != NCS_FP64 && precision != NCS_FP32 && precision != NCS_DF64)
      throw Fail{NCS_E_INPUT, "precision must be FP64, DF64 or FP32"};
    check_ready(c);
    cudaStream_t s = (cudaStream_t)stream;
    for (auto& e : ev) CU(cudaEventCreate(&e));
    CU(cudaEventRecord(ev[0], s));
    outgoing(c, x, precision, s);
    if (use_tree(c)) {
      ensure_tree(c);
      CU(ncs::launch_tree_field(c->d, c->tdev, c->pc.mode, precision, s, ev + 1));
    } else {
      CU(cudaEventRecord(ev[1], s));
      CU(cudaEventRecord(ev[2], s));
      CU(cudaEventRecord(ev[3], s));
      CU(ncs::launch_direct_field(c->d, c->pc.mode, precision, c->pc.eps, s));
      CU(cudaEventRecord(ev[4], s));
      CU(cudaEventRecord(ev[5], s));
    }
    apply_P(c, x, y, precision, s);
    CU(cudaEventRecord(ev[6], s));
    CU(cudaEventSynchronize(ev[6]));
    check_tc(c);
    // stages: outgoing, P2L, coefficients, direct, L2P, apply P, total
    float t[7];
    for (int k = 0; k < 6; ++k) CU(cudaEventElapsedTime(&t[k], ev[k], ev[k + 1]));
    CU(cudaEventElapsedTime(&t[6], ev[0], ev[6]));
    for (int k = 0; k < n && k < 7; ++k) ms[k] = t[k];
  } catch (const Fail& f) {
    rc = finish(c, f);
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  return rc;
}

int ncs_matvec(ncs_ctx* c, const double* x, double* y, int precision) {
  if (c && precision == NCS_PRECISION_DEFAULT) precision = c->precision == NCS_MIXED ? NCS_FP32 : c->precision;
  try {
    if (!c) throw Fail{NCS_E_INPUT, "null context"};
    if (!x || !y) throw Fail{NCS_E_INPUT, "NULL vector"};
    if (precision != NCS_FP64 && precision != NCS_FP32 && precision != NCS_DF64)
      throw Fail{NCS_E_INPUT, "precision must be FP64, DF64 or FP32"};
    check_ready(c);
    ensure_krylov(c, 1);
    const int64_t n = c->d.N * c->d.K;
    CU(cudaMemcpyAsync(c->work, x, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    matvec(c, c->work, c->work + n, precision, c->stream);
    CU(cudaMemcpyAsync(y, c->work + n, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    check_tc(c);
    return NCS_OK;
  } catch (const Fail& f) {
    return finish(c, f);
  } catch (const std::exception& e) {
    return finish(c, Fail{NCS_E_INPUT, e.what()});
  }
}

int ncs_solve(ncs_ctx* c, double tol, int precision, double* fhat, double* scalar, double* Isigma, int* iterations,
              double* relres) {
  if (c && precision == NCS_PRECISION_DEFAULT) precision = c->precision;
  try {
    if (!c) throw Fail{NCS_E_INPUT, "null context"};
    if (!(tol > 0.0 && tol < 1.0)) throw Fail{NCS_E_INPUT, "tol must be in (0, 1)"};
    if (precision != NCS_FP64 && precision != NCS_FP32 && precision != NCS_MIXED && precision != NCS_DF64)
      throw Fail{NCS_E_INPUT, "bad precision"};
    check_ready(c);
    const auto t_start = std::chrono::steady_clock::now();
    for (double& v : c->solve_stats) v = 0.0;
    const int maxit = c->prm.gmres_maxit;
    ensure_krylov(c, maxit);
    const int64_t n = c->d.N * c->d.K;
    cudaStream_t s = c->stream;
    double* b = c->work;           // right-hand side P 1
    double* x = c->work + n;       // solution
    double* r = c->work + 2 * n;   // residual / correction
    // b_i = P 1 for every patch (eq. opinteqnsdisc)
    {
      std::vector<double> P1(c->d.K, 0.0);
      for (int j = 0; j < c->d.K; ++j)
        for (int q = 0; q < c->d.Kstar; ++q) P1[j] += c->pc.P[(size_t)j * c->d.Kstar + q];
      std::vector<double> bh((size_t)n);
      for (int64_t i = 0; i < c->d.N; ++i) std::memcpy(&bh[(size_t)i * c->d.K], P1.data(), c->d.K * sizeof(double));
      CU(cudaMemcpyAsync(b, bh.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
      CU(cudaStreamSynchronize(s));
    }
    const double bnorm = std::sqrt(dev_dot(c, b, b, s));
    int total = 0;
    double est = 1.0, rel = 1.0;
    bool converged = false;
    if (precision != NCS_MIXED) {
      total = gmres(c, b, x, tol, precision, maxit, &est, s);
      // true residual r = b - A x
      matvec(c, x, r, precision, s);
      CU(ncs::launch_axpby(n, 1.0, b, -1.0, r, s));
      rel = std::sqrt(dev_dot(c, r, r, s)) / bnorm;
      ++total;
      c->solve_stats[1] += 1.0;
      c->solve_stats[7] = 1.0;
      // both the GMRES estimate and the recomputed residual must meet the tolerance (an
      // FP32 product's estimate can fall below it while b - A x stays near 1e-6)
      converged = est <= tol && rel <= tol;
    } else {
      // iterative refinement: FP32 inner GMRES, FP64-accurate residuals. Once the
      // residual is small, the correction is small as well and the new residual is
      // updated as r - A corr with the FP32 product: its error (about 1e-6 |A corr|,
      // |A corr| ~ |r|) is then below kUpdateRel * 1e-6 of |b|, far under the tolerance.
      // An updated residual that meets the tolerance is checked by recomputing b - A x at
      // the residual precision before the solve reports convergence.
      constexpr double kUpdateRel = 1e-4;
      double* corr = c->work + 4 * n;
      // the inner solves and the FP32 residual update run on the inner tree (if any); the
      // flag is cleared again on every exit
      if (use_tree(c)) ensure_inner_tree(c);
      struct InnerScope {
        ncs_ctx* c;
        explicit InnerScope(ncs_ctx* cc) : c(cc) { c->inner_active = true; }
        ~InnerScope() { c->inner_active = false; }
      };
      CU(cudaMemsetAsync(x, 0, n * sizeof(double), s));
      CU(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      rel = 1.0;
      bool updated = false;  // r was formed by the FP32 update, not recomputed
      for (int outer = 0; outer < 20; ++outer) {
        if (rel <= tol) {
          if (!updated) break;
          matvec(c, x, r, c->prm.mixed_residual, s);
          CU(ncs::launch_axpby(n, 1.0, b, -1.0, r, s));
          ++total;
          c->solve_stats[1] += 1.0;
          updated = false;
          rel = std::sqrt(dev_dot(c, r, r, s)) / bnorm;
          if (log_level() > 0) std::fprintf(stderr, "ncs: refinement check relres %.3e\n", rel);
          if (!std::isfinite(rel)) throw Fail{NCS_E_NUMERIC, "refinement: non-finite residual"};
          if (rel <= tol) break;
        }
        const double inner_tol = std::max(0.3 * tol / rel, 3e-6);
        double inner_est = 1.0;
        {
          InnerScope in(c);
          total += gmres(c, r, corr, std::min(inner_tol, 0.5), NCS_FP32, maxit, &inner_est, s);
        }
        c->solve_stats[3] += 1.0;
        CU(ncs::launch_axpby(n, 1.0, corr, 1.0, x, s));
        if (rel <= kUpdateRel && c->prm.residual_update) {
          double* Ac = c->work + 3 * n;
          {
            InnerScope in(c);
            matvec(c, corr, Ac, NCS_FP32, s);
          }
          CU(ncs::launch_axpby(n, -1.0, Ac, 1.0, r, s));
          c->solve_stats[2] += 1.0;
          updated = true;
        } else {
          matvec(c, x, r, c->prm.mixed_residual, s);
          CU(ncs::launch_axpby(n, 1.0, b, -1.0, r, s));
          c->solve_stats[1] += 1.0;
          updated = false;
        }
        ++total;
        const double newrel = std::sqrt(dev_dot(c, r, r, s)) / bnorm;
        if (log_level() > 0) std::fprintf(stderr, "ncs: refinement %d relres %.3e\n", outer, newrel);
        if (!std::isfinite(newrel)) throw Fail{NCS_E_NUMERIC, "refinement: non-finite residual"};
        const bool stalled = newrel > 0.9 * rel && outer > 0;
        rel = newrel;
        if (stalled && !(rel <= tol && updated)) break;
      }
      converged = rel <= tol && !updated;
      c->solve_stats[7] = updated ? 0.0 : 1.0;
    }
    c->solve_stats[4] = rel;
    // I_sigma = I . sum_i f_i (eq. getI), then mu or C
    CU(ncs::launch_periodic_dot(n, c->d.K, x, c->d.I, c->partial, c->hdev, s));
    double Is = 0.0;
    CU(cudaMemcpyAsync(&Is, c->hdev, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (fhat) CU(cudaMemcpyAsync(fhat, x, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    check_tc(c);
    c->solve_stats[6] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (Isigma) *Isigma = Is;
    if (scalar) *scalar = (c->pc.mode == NCS_INTERIOR) ? 1.0 / (3.0 * Is) - 0.6 : 4.0 * M_PI * Is;
    if (iterations) *iterations = total;
    if (relres) *relres = rel;
    if (!converged) throw Fail{NCS_E_NOCONV, "GMRES: tolerance not reached within the iteration cap"};
    return NCS_OK;
  } catch (const Fail& f) {
    return finish(c, f);
  } catch (const std::exception& e) {
    return finish(c, Fail{NCS_E_INPUT, e.what()});
  }
}

// Device copies of the one-patch data that the near-patch quadrature needs (uploaded at
// the first evaluation with a target near a patch).
void ensure_near_data(ncs_ctx* c) {
  if (c->near_ready) return;
  const ncs::Precomputed& pc = c->pc;
  const int npan = c->prm.npan, nord = c->prm.nord, nrad = npan * nord;
  if ((int)pc.trad.size() != nrad) throw Fail{NCS_E_STATE, "near-patch evaluation: no one-patch data"};
  const double eps = pc.eps;
  std::vector<double> edges(npan + 1);
  edges[0] = 0.0;
  for (int j = 1; j < npan; ++j) edges[j] = (1.0 - std::ldexp(1.0, -j)) * eps;
  edges[npan] = eps;
  std::vector<double> xn(nrad), bw(nrad), gap(nrad);
  for (int p = 0; p < npan; ++p) {
    const double mid = 0.5 * (edges[p] + edges[p + 1]), half = 0.5 * (edges[p + 1] - edges[p]);
    for (int l = 0; l < nord; ++l) xn[p * nord + l] = (pc.trad[p * nord + l] - mid) / half;
    for (int l = 0; l < nord; ++l) {
      double prod = 1.0;
      for (int m = 0; m < nord; ++m)
        if (m != l) prod *= xn[p * nord + l] - xn[p * nord + m];
      bw[p * nord + l] = 1.0 / prod;
      gap[p * nord + l] = std::sqrt(std::max(0.0, eps - pc.trad[p * nord + l]));
    }
  }
  std::vector<double> g10, w10, g20, w20, tab;
  std::vector<int> off;
  ncs::gauss_legendre(10, g10, w10);
  ncs::gauss_legendre(20, g20, w20);
  ncs::near_phi_tables(tab, off);
  std::vector<double> all;
  auto put = [&all](const std::vector<double>& v) {
    const size_t o = all.size();
    all.insert(all.end(), v.begin(), v.end());
    return o;
  };
  const size_t o_edges = put(edges), o_xn = put(xn), o_bw = put(bw), o_tr = put(pc.trad), o_gap = put(gap),
               o_beta = put(pc.beta), o_g10 = put(g10), o_w10 = put(w10), o_g20 = put(g20), o_w20 = put(w20),
               o_tab = put(tab);
  std::vector<int> ia;
  ia.insert(ia.end(), pc.bm.begin(), pc.bm.end());
  ia.insert(ia.end(), pc.bc.begin(), pc.bc.end());
  ia.insert(ia.end(), off.begin(), off.end());
  ia.push_back(0);  // error flag
  c->near_d = dev_upload(all);
  c->near_i = dev_upload(ia);
  ncs::NearEvalArgs& a = c->near_args;
  const double* b = c->near_d;
  a.K = pc.K;
  a.M = pc.M;
  a.npan = npan;
  a.nord = nord;
  a.eps = eps;
  a.edges = b + o_edges;
  a.xnode = b + o_xn;
  a.bary = b + o_bw;
  a.trad = b + o_tr;
  a.sqrt_gap = b + o_gap;
  a.beta = b + o_beta;
  a.g10 = b + o_g10;
  a.w10 = b + o_w10;
  a.g20 = b + o_g20;
  a.w20 = b + o_w20;
  a.phi_tab = b + o_tab;
  a.bm = c->near_i;
  a.bc = c->near_i + pc.K;
  a.phi_off = c->near_i + 2 * pc.K;
  a.err = c->near_i + 2 * pc.K + (int)off.size();
  c->near_ready = true;
}

int ncs_eval(ncs_ctx* c, int64_t M, const double* targets, const double* fhat, double* out) {
  try {
    check_ready(c);
    if (M < 0 || (M > 0 && (!targets || !out)) || !fhat) throw Fail{NCS_E_INPUT, "bad eval arguments"};
    const double eps = c->pc.eps;
    const int64_t N = c->d.N;
    // patches whose projected geodesic distance from a target is below kNear eps are
    // integrated directly (near-patch quadrature); the others by their skeletons
    constexpr double kNear = 2.5;
    const double h = 2.0 * std::sin(0.5 * kNear * eps);  // chord of kNear eps
    std::unordered_map<uint64_t, std::vector<int>> cells;
    auto key = [h](double x, double y, double z) {
      const int64_t a = (int64_t)std::floor(x / h) + (1 << 20), b = (int64_t)std::floor(y / h) + (1 << 20),
                    cc = (int64_t)std::floor(z / h) + (1 << 20);
      return ((uint64_t)a << 42) ^ ((uint64_t)b << 21) ^ (uint64_t)cc;
    };
    for (int64_t j = 0; j < N; ++j) cells[key(c->centres[3 * j], c->centres[3 * j + 1], c->centres[3 * j + 2])].push_back((int)j);
    std::vector<int64_t> skip_off(M + 1, 0), pair_t;
    std::vector<int> skip_idx;
    for (int64_t t = 0; t < M; ++t) {
      const double* x = targets + 3 * t;
      const double r = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
      if (!(r > 0.0) || !std::isfinite(r)) throw Fail{NCS_E_INPUT, "bad target"};
      if (c->pc.mode == NCS_EXTERIOR && r < 1.0 - 1e-12) throw Fail{NCS_E_INPUT, "exterior target inside the sphere"};
      if (c->pc.mode == NCS_INTERIOR && r > 1.0 + 1e-12) throw Fail{NCS_E_INPUT, "interior target outside the sphere"};
      const double u[3] = {x[0] / r, x[1] / r, x[2] / r};
      for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dz = -1; dz <= 1; ++dz) {
            auto it = cells.find(key(u[0] + dx * h, u[1] + dy * h, u[2] + dz * h));
            if (it == cells.end()) continue;
            for (int j : it->second) {
              const double* cc = &c->centres[3 * j];
              const double cr[3] = {u[1] * cc[2] - u[2] * cc[1], u[2] * cc[0] - u[0] * cc[2], u[0] * cc[1] - u[1] * cc[0]};
              const double g = std::atan2(std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]),
                                          u[0] * cc[0] + u[1] * cc[1] + u[2] * cc[2]);
              if (g >= kNear * eps) continue;
              if (std::fabs(r - 1.0) < 1e-12 && g <= eps * (1.0 + 1e-12))
                throw Fail{NCS_E_INPUT, "target " + std::to_string(t) + " lies on patch " + std::to_string(j) +
                                            " (the potential there is the boundary data)"};
              skip_idx.push_back(j);
              pair_t.push_back(t);
            }
          }
      skip_off[t + 1] = (int64_t)skip_idx.size();
    }
    const int64_t npairs = (int64_t)skip_idx.size();
    if (npairs > 0) {
      if (c->from_operator) throw Fail{NCS_E_INPUT, "targets within 2.5 eps of a patch need the one-patch data (a context from ncs_create)"};
      if (c->pc.M > 31) throw Fail{NCS_E_INPUT, "near-patch evaluation supports Zernike degrees M <= 31"};
      ensure_near_data(c);
    }
    const int64_t n = c->d.N * c->d.K;
    ensure_krylov(c, 1);
    cudaStream_t s = c->stream;
    double *dt = nullptr, *dout = nullptr;
    int64_t* dso = nullptr;
    int64_t* dpt = nullptr;
    int* dsi = nullptr;
    auto release = [&]() {
      cudaFree(dt);
      cudaFree(dout);
      cudaFree(dso);
      cudaFree(dpt);
      cudaFree(dsi);
    };
    try {
      dt = dev_alloc<double>(std::max<int64_t>(1, 3 * M));
      dout = dev_alloc<double>(std::max<int64_t>(1, M));
      dso = dev_upload(skip_off);
      dpt = dev_upload(pair_t);
      dsi = dev_upload(skip_idx);
      CU(cudaMemcpyAsync(c->work, fhat, n * sizeof(double), cudaMemcpyHostToDevice, s));
      if (M) CU(cudaMemcpyAsync(dt, targets, 3 * M * sizeof(double), cudaMemcpyHostToDevice, s));
      CU(ncs::launch_outgoing(c->d, c->work, NCS_FP64, s));
      CU(ncs::launch_eval_skip(c->d, c->pc.mode, M, dt, dout, npairs ? dso : nullptr, npairs ? dsi : nullptr, s));
      int nerr = 0;
      if (npairs > 0) {
        ncs::NearEvalArgs a = c->near_args;
        a.pair_target = dpt;
        a.pair_patch = dsi;
        a.targets = dt;
        a.centres = c->d.centres;
        a.fhat = c->work;
        a.out = dout;
        CU(cudaMemsetAsync(a.err, 0, sizeof(int), s));
        CU(ncs::launch_near_eval(a, c->pc.mode, npairs, s));
        CU(cudaMemcpyAsync(&nerr, a.err, sizeof(int), cudaMemcpyDeviceToHost, s));
      }
      CU(ncs::launch_periodic_dot(n, c->d.K, c->work, c->d.I, c->partial, c->hdev, s));
      double Is = 0.0;
      CU(cudaMemcpyAsync(&Is, c->hdev, sizeof(double), cudaMemcpyDeviceToHost, s));
      if (M) CU(cudaMemcpyAsync(out, dout, M * sizeof(double), cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      if (nerr) throw Fail{NCS_E_INPUT, "near-patch evaluation: a target too close to a patch for the radial rule"};
      for (int64_t t = 0; t < M; ++t) {
        const double* x = targets + 3 * t;
        const double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
        if (c->pc.mode == NCS_EXTERIOR)
          out[t] = 1.0 - out[t];  // ubar = 1 - u (Section 2.2)
        else
          out[t] = (out[t] - 1.0) / (3.0 * (-Is)) + (1.0 - r2) / 6.0;  // eq. (vtilde), D = -I_sigma
      }
    } catch (...) {
      release();
      throw;
    }
    release();
    return NCS_OK;
  } catch (const Fail& f) {
    return finish(c, f);
  } catch (const std::exception& e) {
    return finish(c, Fail{NCS_E_INPUT, e.what()});
  }
}

int ncs_patch_residual(ncs_ctx* c, int64_t i, const double* fhat, int nt, int nth, double* rms) {
  try {
    if (!c || !fhat || !rms) throw Fail{NCS_E_INPUT, "bad residual arguments"};
    check_ready(c);
    if (i < 0 || i >= c->d.N) throw Fail{NCS_E_INPUT, "patch index out of range"};
    const ncs::Precomputed& pc = c->pc;
    if (nt <= 0) nt = pc.M + 8;
    if (nth <= 0) nth = 2 * pc.M + 10;
    if (nt > 4096 || nth > 8192) throw Fail{NCS_E_INPUT, "residual grid too large"};
    const double eps = pc.eps;
    const int K = pc.K;
    // the patch's frame (the one of its Zernike nodes and skeletons): e1 = z x c / |z x c|
    // (x at the poles), e2 = c x e1
    const double* cc = &c->centres[3 * i];
    double e1[3] = {-cc[1], cc[0], 0.0};
    const double na2 = e1[0] * e1[0] + e1[1] * e1[1];
    if (na2 >= 1e-24) {
      const double inv = 1.0 / std::sqrt(na2);
      e1[0] *= inv;
      e1[1] *= inv;
    } else {
      e1[0] = 1.0;
      e1[1] = 0.0;
    }
    const double e2[3] = {cc[1] * e1[2] - cc[2] * e1[1], cc[2] * e1[0] - cc[0] * e1[2],
                          cc[0] * e1[1] - cc[1] * e1[0]};
    std::vector<double> gx, gw;
    ncs::gauss_legendre(nt, gx, gw);
    const int64_t M = (int64_t)nt * nth;
    std::vector<double> tg(3 * (size_t)M), dA(M), selfv(M);
    const double* fi = fhat + (size_t)i * K;
    std::vector<double> rad(K);
    for (int a = 0; a < nt; ++a) {
      const double t = 0.5 * eps * (gx[a] + 1.0), wt = 0.5 * eps * gw[a];
      const double st = std::sin(t), ct = std::cos(t);
      for (int k = 0; k < K; ++k) {
        const double nn = (pc.bm[k] == 0 ? 2.0 : 1.0) * ncs::kPi / (2.0 * pc.bn[k] + 2.0);  // eq. zorthog
        rad[k] = fi[k] * ncs::zernike_radial(pc.bn[k], pc.bm[k], t / eps) / std::sqrt(nn);
      }
      for (int b = 0; b < nth; ++b) {
        const double th = 2.0 * ncs::kPi * b / nth, ch = std::cos(th), sh = std::sin(th);
        const int64_t q = (int64_t)a * nth + b;
        for (int k = 0; k < 3; ++k) tg[3 * q + k] = ct * cc[k] + st * (ch * e1[k] + sh * e2[k]);
        dA[q] = wt * st * 2.0 * ncs::kPi / nth;
        double v = 0.0;
        for (int k = 0; k < K; ++k) v += rad[k] * (pc.bc[k] ? std::sin(pc.bm[k] * th) : std::cos(pc.bm[k] * th));
        selfv[q] = v;
      }
    }
    const int64_t n = c->d.N * c->d.K;
    ensure_krylov(c, 1);
    cudaStream_t s = c->stream;
    double *dt = nullptr, *dout = nullptr;
    std::vector<double> u(M);
    try {
      CU(cudaMalloc(&dt, 3 * (size_t)M * sizeof(double)));
      CU(cudaMalloc(&dout, (size_t)M * sizeof(double)));
      CU(cudaMemcpyAsync(c->work, fhat, n * sizeof(double), cudaMemcpyHostToDevice, s));
      CU(cudaMemcpyAsync(dt, tg.data(), 3 * (size_t)M * sizeof(double), cudaMemcpyHostToDevice, s));
      CU(ncs::launch_outgoing(c->d, c->work, NCS_FP64, s));
      CU(ncs::launch_eval(c->d, pc.mode, M, dt, dout, s, i));  // patch i left out
      CU(cudaMemcpyAsync(u.data(), dout, (size_t)M * sizeof(double), cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
    } catch (...) {
      cudaFree(dt);
      cudaFree(dout);
      throw;
    }
    cudaFree(dt);
    cudaFree(dout);
    double num = 0.0, den = 0.0;
    for (int64_t q = 0; q < M; ++q) {
      const double r = selfv[q] + u[q] - 1.0;
      num += dA[q] * r * r;
      den += dA[q];
    }
    *rms = std::sqrt(num / den);
    return NCS_OK;
  } catch (const Fail& f) {
    return finish(c, f);
  } catch (const std::bad_alloc&) {
    return finish(c, Fail{NCS_E_OOM, "out of host memory"});
  } catch (const std::exception& e) {
    return finish(c, Fail{NCS_E_INPUT, e.what()});
  }
}

int ncs_block_dots(int64_t n, int k, const double* V, int64_t ld, const double* w, double* out, void* stream) {
  if (n < 0 || k < 0 || ld < n || (k > 0 && (!V || !w || !out))) return NCS_E_INPUT;
  if (k == 0) return NCS_OK;
  double* partial = nullptr;
  if (cudaMalloc(&partial, (size_t)ncs::kDotChunks * k * sizeof(double)) != cudaSuccess) return NCS_E_OOM;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = NCS_OK;
  if (ncs::launch_dots(n, k, V, ld, w, partial, out, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    rc = NCS_E_CUDA;
  cudaFree(partial);
  return rc;
}

int ncs_tc_gemm_f32(int64_t rows, int cols, int kdim, const float* A, const float* B, float* D, void* stream) {
  if (rows < 0 || cols < 0 || kdim < 1 || !A || !B || !D) return NCS_E_INPUT;
  if (rows == 0 || cols == 0) return NCS_OK;
  int* err = nullptr;
  uint32_t *pack = nullptr, *apack = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return NCS_E_OOM;
  if (cudaMalloc(&pack, (size_t)ncs::tc_pack_words(cols, kdim, ncs::tc_block_cols(cols)) * sizeof(uint32_t)) !=
          cudaSuccess ||
      cudaMalloc(&apack, (size_t)ncs::tc_pack_words(rows, kdim, 128) * sizeof(uint32_t)) != cudaSuccess) {
    cudaFree(pack);
    cudaFree(err);
    return NCS_E_OOM;
  }
  int rc = NCS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess ||
      ncs::launch_tc_pack_b(B, cols, kdim, pack, s) != cudaSuccess ||
      ncs::launch_tc_gemm_f32(rows, cols, kdim, A, apack, pack, D, err, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    rc = NCS_E_CUDA;
  } else {
    int f = 0;
    if (cudaMemcpy(&f, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = NCS_E_CUDA;
    else if (f) rc = NCS_E_TIMEOUT;
  }
  cudaFree(apack);
  cudaFree(pack);
  cudaFree(err);
  return rc;
}

int ncs_batch_solve(int B, const double* eps, const int* mode, const int64_t* N, const double* const* centres,
                    int K, double tol, int precision, const ncs_params* params, int workers, double* scalar,
                    double* Isigma, int* iterations, double* relres, int* status, double* seconds) {
  if (B < 1 || !eps || !mode || !N || !centres || K < 1 || !(tol > 0.0 && tol < 1.0)) return NCS_E_INPUT;
  if (precision != NCS_FP64 && precision != NCS_FP32 && precision != NCS_MIXED && precision != NCS_DF64)
    return NCS_E_INPUT;
  for (int b = 0; b < B; ++b)
    if (!centres[b] || N[b] < 1 || !(eps[b] > 0.0 && eps[b] < 1.0) || (mode[b] != 0 && mode[b] != 1))
      return NCS_E_INPUT;
  ncs_params prm;
  if (params)
    prm = *params;
  else
    ncs_default_params(&prm);
  const bool user_graphs = prm.cuda_graphs != 0;  // the grouped solve runs alone: it may capture
  prm.threads = 1;  // one host thread per instance; instances run concurrently
  // no CUDA-graph capture: a capture on one worker's stream makes device-wide
  // synchronisation (which allocation, freeing and the precompute of the other workers may
  // imply) invalid until it ends; the instances' steps are launched directly
  prm.cuda_graphs = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NCS_E_CUDA;
  unsigned hw = std::thread::hardware_concurrency();
  int W = workers > 0 ? workers : (int)std::max(1u, hw);
  W = std::min(W, B);
  std::atomic<int> next(0);
  std::atomic<double> t_pre(0.0), t_solve(0.0);
  // spheres below the tree threshold are set up by the workers and solved together
  // afterwards (one grouped system per mode), when the solve is mixed
  std::mutex small_mu;
  std::vector<ncs_ctx*> small_ctx;
  std::vector<int> small_idx;
  auto add_time = [](std::atomic<double>& a, double v) {
    double cur = a.load();
    while (!a.compare_exchange_weak(cur, cur + v)) {
    }
  };
  const auto t0 = std::chrono::steady_clock::now();
  auto work = [&]() {
    cudaSetDevice(dev);
    for (;;) {
      const int b = next.fetch_add(1);
      if (b >= B) break;
      const auto a0 = std::chrono::steady_clock::now();
      ncs_ctx* c = nullptr;
      ncs_params pb = prm;
      if (prm.batch_ladder_by_n) pb.id_ladder_max = std::min(prm.id_ladder_max, batch_ladder_extent(N[b]));
      const bool grouped = prm.batch_grouped && precision == NCS_MIXED && prm.method != NCS_METHOD_TREE &&
                           N[b] < prm.tree_min_patches;
      if (grouped) pb.method = NCS_METHOD_DIRECT;
      int rc = ncs_create(eps[b], mode[b], K, &pb, &c);
      if (rc == NCS_OK) rc = ncs_set_patches(c, N[b], centres[b]);
      const auto a1 = std::chrono::steady_clock::now();
      if (grouped && rc == NCS_OK) {
        add_time(t_pre, std::chrono::duration<double>(a1 - a0).count());
        std::lock_guard<std::mutex> lk(small_mu);
        small_ctx.push_back(c);
        small_idx.push_back(b);
        continue;
      }
      double sc = 0.0, is = 0.0, rr = 0.0;
      int it = 0;
      if (rc == NCS_OK) rc = ncs_solve(c, tol, precision, nullptr, &sc, &is, &it, &rr);
      const auto a2 = std::chrono::steady_clock::now();
      if (scalar) scalar[b] = sc;
      if (Isigma) Isigma[b] = is;
      if (iterations) iterations[b] = it;
      if (relres) relres[b] = rr;
      if (status) status[b] = rc;
      ncs_destroy(c);
      add_time(t_pre, std::chrono::duration<double>(a1 - a0).count());
      add_time(t_solve, std::chrono::duration<double>(a2 - a1).count());
    }
  };
  std::vector<std::thread> th;
  for (int w = 0; w < W; ++w) th.emplace_back(work);
  for (auto& t : th) t.join();
  if (!small_ctx.empty()) {
    const auto g0 = std::chrono::steady_clock::now();
    cudaStream_t gs = nullptr;
    int grc = cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking) == cudaSuccess ? NCS_OK : NCS_E_CUDA;
    for (int m = 0; m < 2; ++m) {
      std::vector<ncs_ctx*> cs;
      std::vector<int> idx;
      for (size_t q = 0; q < small_ctx.size(); ++q)
        if (mode[small_idx[q]] == m) {
          cs.push_back(small_ctx[q]);
          idx.push_back(small_idx[q]);
        }
      if (cs.empty()) continue;
      std::vector<GroupResult> gr;
      int rc = grc;
      if (rc == NCS_OK) {
        try {
          group_solve(cs, tol, user_graphs, gs, gr);
        } catch (const Fail& f) {
          rc = f.code;
          if (log_level() > 0) std::fprintf(stderr, "ncs: grouped solve: %s\n", f.msg.c_str());
        } catch (const std::exception& e) {
          rc = NCS_E_INPUT;
          if (log_level() > 0) std::fprintf(stderr, "ncs: grouped solve: %s\n", e.what());
        }
      }
      for (size_t q = 0; q < idx.size(); ++q) {
        const int b = idx[q];
        const GroupResult o = rc == NCS_OK ? gr[q] : GroupResult{0.0, 0.0, 1.0, 0, rc};
        if (scalar) scalar[b] = o.scalar;
        if (Isigma) Isigma[b] = o.Is;
        if (iterations) iterations[b] = o.iters;
        if (relres) relres[b] = o.rel;
        if (status) status[b] = o.status;
      }
    }
    if (gs) cudaStreamDestroy(gs);
    for (ncs_ctx* c : small_ctx) ncs_destroy(c);
    add_time(t_solve, std::chrono::duration<double>(std::chrono::steady_clock::now() - g0).count());
  }
  const double total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (seconds) {
    seconds[0] = t_pre.load();    // summed over instances (set-up: precompute + tree)
    seconds[1] = t_solve.load();  // summed over instances
    seconds[2] = total;           // wall clock of the whole batch
  }
  if (status)
    for (int b = 0; b < B; ++b)
      if (status[b] != NCS_OK) return status[b];
  return NCS_OK;
}

int ncs_set_tuning(ncs_ctx* c, const ncs_tuning* t) {
  if (!c || !t) return NCS_E_INPUT;
  if (!tuning_valid(*t)) return finish(c, Fail{NCS_E_INPUT, "ncs_set_tuning: value out of range"});
  if (c->device_ready) cudaSetDevice(c->device);
  apply_tuning(c, *t);
  return NCS_OK;
}

int ncs_get_tuning(const ncs_ctx* c, ncs_tuning* t) {
  if (!c || !t) return NCS_E_INPUT;
  *t = c->tune;
  return NCS_OK;
}

int ncs_tune(ncs_ctx* c, int flags, const char* cache_path, ncs_tuning* out, double* report, int nrep) {
  double* buf = nullptr;
  cudaEvent_t ev[6] = {};
  int rc = NCS_OK;
  try {
    if (!c) throw Fail{NCS_E_INPUT, "null context"};
    if (flags < 1 || flags > 3) throw Fail{NCS_E_INPUT, "ncs_tune: flags must be 1, 2 or 3"};
    check_ready(c);
    if (!use_tree(c)) throw Fail{NCS_E_STATE, "ncs_tune: the context does not use the tree method"};
    ensure_tree(c);
    const auto t_start = std::chrono::steady_clock::now();
    cudaStream_t s = c->stream;
    double rep[6] = {0, 0, 0, 0, 0, 0};
    const std::string key = tune_key(c);
    ncs_tuning best = c->tune;
    if (cache_path && tune_cache_lookup(cache_path, key, &best)) {
      apply_tuning(c, best);
      rep[5] = 1.0;
    } else {
      const int64_t n = c->d.N * c->d.K, nz = c->d.N * c->d.Kstar;
      buf = dev_alloc<double>((size_t)(n + 2 * nz + 2));
      double *x = buf, *zref = buf + n, *zt = buf + n + nz, *md = buf + n + 2 * nz;
      {
        // a fixed pseudo-random input (splitmix64 to [-1, 1))
        std::vector<double> xh((size_t)n);
        uint64_t st = 0x9e3779b97f4a7c15ull;
        for (auto& v : xh) {
          uint64_t z = (st += 0x9e3779b97f4a7c15ull);
          z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
          z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
          z ^= z >> 31;
          v = 2.0 * (double)(z >> 11) * (1.0 / 9007199254740992.0) - 1.0;
        }
        CU(cudaMemcpyAsync(x, xh.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
        field(c, x, NCS_DF64, s);
        CU(cudaMemcpyAsync(zref, c->d.z, nz * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CU(cudaStreamSynchronize(s));
      }
      for (auto& e : ev) CU(cudaEventCreate(&e));
      int trials = 0;
      // FP32 field of x under the current configuration: min over reps of the P2L and
      // direct-list stage times and of the whole field, and its error against zref
      struct Meas {
        double p2l, direct, total, err;
      };
      auto measure = [&](int reps) {
        ensure_tree(c);
        Meas m{1e300, 1e300, 1e300, 0.0};
        for (int r = 0; r <= reps; ++r) {
          CU(cudaEventRecord(ev[5], s));
          outgoing(c, x, NCS_FP32, s);
          CU(ncs::launch_tree_field(c->d, c->tdev, c->pc.mode, NCS_FP32, s, ev));
          CU(cudaEventSynchronize(ev[4]));
          ++trials;
          if (r == 0) continue;  // warm-up
          float a = 0, b = 0, t = 0;
          CU(cudaEventElapsedTime(&a, ev[0], ev[1]));
          CU(cudaEventElapsedTime(&b, ev[2], ev[3]));
          CU(cudaEventElapsedTime(&t, ev[5], ev[4]));
          m.p2l = std::min(m.p2l, (double)a);
          m.direct = std::min(m.direct, (double)b);
          m.total = std::min(m.total, (double)t);
        }
        CU(ncs::launch_maxabs_diff(nz, c->d.z, zref, md, s));
        double h[2];
        CU(cudaMemcpyAsync(h, md, sizeof h, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        check_tc(c);
        m.err = h[0] / std::max(h[1], 1e-300);
        return m;
      };
      constexpr double kTol = 2e-5;  // the FP32 product's accuracy bar
      constexpr int kReps = 3;
      const ncs_tuning start = c->tune;
      const Meas m0 = measure(kReps);
      rep[0] = m0.total;
      double best_total = m0.err <= kTol ? m0.total : 1e300;
      double best_err = m0.err;
      if (flags & 1) {
        // P2L variants (the direct lists are timed as a separate stage of the same runs)
        double bp = m0.err <= kTol ? m0.p2l : 1e300;
        ncs_tuning bt = start;
        for (int jt : {8, 16})
          for (int poly : {0, 2, 4, 6})
            for (int rsq : {0, 4, 8}) {
              ncs_tuning t = start;
              t.p2l_tile = jt;
              t.p2l_poly = poly;
              t.p2l_rsq = rsq;
              if (!tuning_valid(t) || (jt == start.p2l_tile && poly == start.p2l_poly && rsq == start.p2l_rsq))
                continue;
              apply_tuning(c, t);
              const Meas m = measure(kReps);
              if (m.err <= kTol && m.p2l < bp) bp = m.p2l, bt = t;
            }
        double bd = m0.err <= kTol ? m0.direct : 1e300;
        const ncs_tuning bp2l = bt;
        for (int poly : {0, 2, 4, 6})
          for (int rsq : {0, 4, 8}) {
            ncs_tuning t = bp2l;
            t.direct_poly = poly;
            t.direct_rsq = rsq;
            if (!tuning_valid(t) || (poly == start.direct_poly && rsq == start.direct_rsq)) continue;
            apply_tuning(c, t);
            const Meas m = measure(kReps);
            if (m.err <= kTol && m.direct < bd) bd = m.direct, bt.direct_poly = poly, bt.direct_rsq = rsq;
          }
        apply_tuning(c, bt);
        const Meas m = measure(kReps);
        best = bt;
        best_total = m.err <= kTol ? m.total : 1e300;
        best_err = m.err;
        if (!(m.err <= kTol)) {  // keep the starting configuration
          best = start;
          best_total = m0.total;
          best_err = m0.err;
        }
        apply_tuning(c, best);
      }
      if (flags & 2) {
        // work-item size and grid-or-direct weight: each candidate on its own tree
        const ncs_tuning base = best;
        for (int ip : {16, 32})
          for (double w : {0.05, 0.1, 0.2}) {
            ncs_tuning t = base;
            t.item_patches = ip;
            t.l2p_weight = w;
            if (!tuning_valid(t) || (ip == base.item_patches && w == base.l2p_weight)) continue;
            apply_tuning(c, t);
            const Meas m = measure(kReps);
            if (m.err <= kTol && m.total < best_total) best_total = m.total, best = t, best_err = m.err;
          }
        apply_tuning(c, best);
      }
      rep[1] = best_total;
      rep[2] = trials;
      rep[3] = best_err;
      if (cache_path) tune_cache_store(cache_path, key, best);
    }
    rep[4] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (out) *out = c->tune;
    for (int i = 0; report && i < nrep && i < 6; ++i) report[i] = rep[i];
  } catch (const Fail& f) {
    rc = finish(c, f);
  } catch (const std::bad_alloc&) {
    rc = finish(c, Fail{NCS_E_OOM, "out of host memory"});
  } catch (const std::exception& e) {
    rc = finish(c, Fail{NCS_E_INPUT, e.what()});
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (buf) cudaFree(buf);
  return rc;
}

int ncs_solve_stats(const ncs_ctx* c, double* out, int n) {
  if (!c || !out) return NCS_E_INPUT;
  for (int i = 0; i < n && i < 8; ++i) out[i] = c->solve_stats[i];
  return NCS_OK;
}

const char* ncs_last_error(const ncs_ctx* c) { return c ? c->err.c_str() : g_static_err; }

int64_t ncs_launch_count(void) { return (int64_t)ncs::g_launches.load(std::memory_order_relaxed); }

void ncs_destroy(ncs_ctx* c) {
  if (!c) return;
  if (c->device_ready) cudaSetDevice(c->device);
  free_all(c);
  delete c;
}

}  // extern "C"
