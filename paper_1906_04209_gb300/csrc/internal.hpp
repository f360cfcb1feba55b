// Internal declarations shared by the host API and the CUDA launchers.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "ncs.h"
#include "precompute.hpp"
#include "tree.hpp"

namespace ncs {

// Process-wide number of kernels the library has launched (read by ncs_launch_count).
// Every launch site is written `count_launch(), kernel<<<...>>>(...)`.
extern std::atomic<long long> g_launches;
inline void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Device-resident data of one patch layout plus the precompute.
struct DeviceData {
  int K = 0, Kstar = 0;
  int p = 0;                   // skeleton points over all representations (p_total)
  int nrep = 0;                // outgoing representations (increasing far-field radius)
  int pmax = 0;                // largest p_k
  int p0 = 0;                  // p of representation 0 (far field beyond 2 eps)
  int* rep_p = nullptr;        // nrep: p_k
  int* rep_off = nullptr;      // nrep: column offset of representation k
  double* rep_rho = nullptr;   // nrep: far-field radius (geodesic) of representation k
  int64_t N = 0;
  double* centres = nullptr;   // N*3
  double* zloc = nullptr;      // Kstar*3 local offsets of the Zernike nodes
  double* sloc = nullptr;      // p*3 local offsets of the skeleton points (all representations)
  double* TT64 = nullptr;      // K*p, all T_k stacked and transposed
  float* TT32 = nullptr;
  double* PT64 = nullptr;      // Kstar*K, P transposed
  float* PT32 = nullptr;
  double* soff64 = nullptr;    // N*p*3 skeleton offsets (global frame) from each centre
  float* soff32 = nullptr;
  double* rho64 = nullptr;     // N*p outgoing coefficients
  float* rho32 = nullptr;
  double* z = nullptr;         // N*Kstar field at the Zernike nodes
  double* I = nullptr;         // K
  float4* logtab = nullptr;    // 64 x (log c hi, lo, 1/c hi, lo), c = 1 + (i + 0.5)/64
  uint32_t* Tpack = nullptr;   // all T_k stacked (p x K), TF32 hi/lo tensor-core blocks
  uint32_t* Ppack = nullptr;   // P (K x Kstar), TF32 hi/lo tensor-core blocks
  uint32_t* Apack = nullptr;   // x or z of one product as TF32 hi/lo blocks (tensor_cores only)
  int* tc_err = nullptr;       // set by a tensor-core kernel whose bounded wait gave up
};

// ---- launchers (kernels.cu)
cudaError_t launch_skeleton_offsets(const DeviceData& d, cudaStream_t s);
cudaError_t launch_outgoing(const DeviceData& d, const double* x, int prec, cudaStream_t s);
cudaError_t launch_direct_field(const DeviceData& d, int mode, int prec, double eps, cudaStream_t s);
cudaError_t launch_apply_P(const DeviceData& d, const double* x, double* y, int prec, cudaStream_t s);
// Single-layer potential of every patch's finest skeleton representation at M targets
// (off-surface Green's functions); patch `skip` (if >= 0) is left out of the sum.
cudaError_t launch_eval(const DeviceData& d, int mode, int64_t M, const double* targets,
                        double* out, cudaStream_t s, int64_t skip = -1);

// ---- near-patch evaluation (neareval.cu)
constexpr int kNearMaxLevels = 50;
struct NearEvalArgs {
  const int64_t* pair_target;  // npairs: target of each (target, near patch) pair
  const int* pair_patch;       // npairs: the patch
  const double* targets;       // M x 3
  const double* centres;       // N x 3
  const double* fhat;          // N x K densities
  int K = 0, M = 0, npan = 0, nord = 0;
  double eps = 0.0;
  const double* edges;         // npan + 1 radial panel edges
  const double* xnode;         // npan * nord nodes, normalised to [-1, 1] on their panel
  const double* bary;          // npan * nord barycentric weights of those nodes
  const double* trad;          // npan * nord radial nodes t
  const double* sqrt_gap;      // npan * nord: sqrt(eps - t)
  const double* beta;          // (npan * nord) x K radial profiles
  const int* bm;               // K angular orders
  const int* bc;               // K: 1 for sin, 0 for cos
  const double *g10, *w10, *g20, *w20;  // Gauss-Legendre rules on [-1, 1]
  const double* phi_tab;       // (weight, sin^2(phi/2), cos phi) per node
  const int* phi_off;          // kNearMaxLevels + 2 node offsets
  double* out;                 // M: the pair's potential is added atomically
  int* err;                    // set when a radial rule would exceed its shared-memory room
};
void near_phi_tables(std::vector<double>& tab, std::vector<int>& off);
cudaError_t launch_near_eval(const NearEvalArgs& a, int mode, int64_t npairs, cudaStream_t s);
// launch_eval with a per-target list of patches left out (CSR: skip_off[M + 1], skip_idx)
cudaError_t launch_eval_skip(const DeviceData& d, int mode, int64_t M, const double* targets, double* out,
                             const int64_t* skip_off, const int* skip_idx, cudaStream_t s);

// ---- tensor-core GEMMs (tc_gemm.cu)
// Operands of the tensor-core GEMMs as TF32 hi/lo blocks in the shared-memory layout:
// tc_pack_words 32-bit words for nrows x Kd in row tiles of H; B operands (the constant
// operators) use tiles of tc_block_cols(cols) and are packed once by launch_tc_pack_b,
// A operands (x, z) use tiles of 128 and are packed by each GEMM launcher.
int tc_block_cols(int cols);
int64_t tc_pack_words(int64_t nrows, int Kd, int H);
cudaError_t launch_tc_pack_b(const float* B, int cols, int Kd, uint32_t* out, cudaStream_t s);
cudaError_t launch_tc_outgoing(const DeviceData& d, const double* x, int* err, cudaStream_t s);
cudaError_t launch_tc_apply_P(const DeviceData& d, const double* x, double* y, int* err, cudaStream_t s);
cudaError_t launch_tc_gemm_f32(int64_t rows, int cols, int Kd, const float* A, uint32_t* Apack,
                               const uint32_t* Bpack, float* D, int* err, cudaStream_t s);

// ---- dense-vector kernels for GMRES (blas.cu)
cudaError_t launch_dots(int64_t n, int k, const double* V, int64_t ld, const double* w,
                        double* partial, double* out, cudaStream_t s);
cudaError_t launch_sub_combination(int64_t n, int k, const double* V, int64_t ld, const double* h,
                                   double* w, double sign, cudaStream_t s);
cudaError_t launch_scale_copy(int64_t n, const double* w, double a, double* v, cudaStream_t s);
cudaError_t launch_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t s);
cudaError_t launch_nonfinite_count(int64_t n, const double* x, int* out, cudaStream_t s);
// out[0] = max |a_i - b_i|, out[1] = max |b_i| over n entries (out: 2 device doubles, zeroed here)
cudaError_t launch_maxabs_diff(int64_t n, const double* a, const double* b, double* out, cudaStream_t s);
cudaError_t launch_periodic_dot(int64_t n, int K, const double* x, const double* I, double* partial,
                                double* out, cudaStream_t s);
constexpr int kDotChunks = 64;

// ---- GMRES state on the device (blas.cu). The column in progress is m; a step reads it,
// so the same launches (and one captured CUDA graph) serve every iteration.
constexpr int kGmresRunning = 0, kGmresConverged = 1, kGmresHappy = 2, kGmresBreakdown = 3, kGmresNonFinite = 4;
struct GmresState {
  int m;       // Arnoldi columns completed (= index of the column in progress)
  int done;    // 1: no further step (flag says why; flag 0 with done = iteration cap)
  int flag;    // kGmres*
  int maxit;   // iteration cap
  double beta; // |r0|
  double tol;  // relative tolerance of the estimate |g_m| / beta
  double res;  // current estimate
  double hn;   // norm of the newest (orthogonalised) vector
};
// Device pointers of one context's GMRES workspace.
struct GmresDev {
  int maxit = 0;
  GmresState* st = nullptr;
  double* H = nullptr;        // (maxit + 1) x maxit, column-major
  double* cs = nullptr;       // maxit
  double* sn = nullptr;       // maxit
  double* g = nullptr;        // maxit + 1
  double* y = nullptr;        // maxit
  double* h1 = nullptr;       // maxit + 1: first Gram-Schmidt pass
  double* h2 = nullptr;       // maxit + 1: second pass
  double* partial = nullptr;  // kDotChunks x (maxit + 1)
  double* pnorm = nullptr;    // gmres_update_blocks(n)
  double* vk = nullptr;       // n: copy of the newest basis vector (the product's input)
};
int gmres_update_blocks(int64_t n);
// Two Gram-Schmidt passes of w against V_0..V_m, the Givens update of column m and
// V_{m+1} = vk = w / |w| (every launch a no-op once st->done).
cudaError_t launch_arnoldi_orthogonalize(int64_t n, const double* V, double* w, const GmresDev& gd,
                                         cudaStream_t s);
// y = R^-1 g (m from the device state).
cudaError_t launch_gmres_backsolve(const GmresDev& gd, cudaStream_t s);

// ---- grouped solve of small spheres (group.cu): B instances sharing K, Kstar and the
// mode, their patches concatenated (patch i of the group belongs to instance pinst[i];
// instance b owns patches [pbase[b], pbase[b + 1]) and entries [pbase[b] K, pbase[b + 1] K)
// of every vector). Each instance keeps its eps, outgoing operator and GMRES state.
struct GroupDev {
  int B = 0, K = 0, Kstar = 0, mode = 0, maxit = 0, pmax = 0;
  int seg_blocks = 1;              // blocks per instance of the segmented vector kernels
  int64_t P = 0;                   // patches over all instances
  const int* pinst = nullptr;      // P: instance of each patch
  const int64_t* pbase = nullptr;  // B + 1: first patch of each instance
  const int64_t* roff = nullptr;   // P: first outgoing coefficient of each patch
  const int* inst_ptot = nullptr;  // B: skeleton points over all representations
  const int64_t* tt_off = nullptr; // B: offset of the instance's T^T (K x ptot) in TT64/TT32
  const double* inst_eps = nullptr;
  const int* inst_nrep = nullptr;     // B: outgoing representations
  const int* inst_repbase = nullptr;  // B: first entry of the instance in rep_p/rep_off/rep_rho
  const int* rep_p = nullptr;
  const int* rep_off = nullptr;
  const double* rep_rho = nullptr;
  const double* zloc = nullptr;    // B x Kstar x 3 local Zernike-node offsets
  const double* centres = nullptr; // P x 3
  const double* soff64 = nullptr;  // skeleton offsets, laid out like the coefficients (x 3)
  const float* soff32 = nullptr;
  double* rho64 = nullptr;         // outgoing coefficients
  float* rho32 = nullptr;
  const double* TT64 = nullptr;
  const float* TT32 = nullptr;
  double* z = nullptr;             // P x Kstar
  const double* I = nullptr;       // B x K
  const float4* logtab = nullptr;
  GmresState* st = nullptr;        // B
  double *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;  // per instance blocks
  double *h1 = nullptr, *h2 = nullptr;  // B x (maxit + 1)
  double* pnorm = nullptr;         // B x seg_blocks
  double* vk = nullptr;            // P x K: the newest basis vector of every instance
};
int group_seg_blocks(int64_t maxseg);
// z = compressed far field of x (outgoing products, then the direct sums per instance)
cudaError_t launch_group_field(const GroupDev& g, const double* x, int prec, cudaStream_t s);
// One Arnoldi step of every running instance (two Gram-Schmidt passes, Givens, normalise).
cudaError_t launch_group_arnoldi(const GroupDev& g, const double* V, double* w, cudaStream_t s);
// e = V y with y = R^-1 g per instance
cudaError_t launch_group_solution(const GroupDev& g, const double* V, double* e, cudaStream_t s);
// out[b] = a . c over instance b's segment
cudaError_t launch_group_dots(const GroupDev& g, const double* a, const double* c, double* out, cudaStream_t s);
// out[b] = I_b . sum of instance b's densities
cudaError_t launch_group_isigma(const GroupDev& g, const double* x, double* out, cudaStream_t s);
// x[seg_b] *= a[b]
cudaError_t launch_group_scale(const GroupDev& g, const double* a, double* x, cudaStream_t s);

}  // namespace ncs

// The opaque context of the C ABI.
struct ncs_ctx {
  ncs_params prm{};
  int precision = NCS_MIXED;  // used when a call passes NCS_PRECISION_DEFAULT
  ncs::Precomputed pc;
  bool from_operator = false;
  std::string err;
  int device = 0;
  cudaStream_t stream = nullptr;
  std::vector<double> centres;
  int method = NCS_METHOD_AUTO;
  ncs::DeviceData d;
  ncs::TreeHost tree;
  ncs::TreeDevice tdev;
  bool tree_built = false;      // host tree ready
  bool tree_uploaded = false;   // device copy ready
  // the tree of the mixed solve's inner FP32 products: incoming grids to prm.inner_grid_tol
  ncs::TreeHost tree_in;
  ncs::TreeDevice tdev_in;
  bool tree_in_built = false;
  bool tree_in_uploaded = false;
  bool inner_active = false;    // inside ncs_solve's inner solves: FP32 tree products use tdev_in
  bool device_ready = false;    // operator uploaded, stream created
  bool layout_dirty = false;    // centres changed since the last upload
  // GMRES workspace
  double* V = nullptr;
  int Vcap = 0;
  double* work = nullptr;      // 5 vectors of N*K
  double* partial = nullptr;   // kDotChunks * (maxit+2)
  double* hdev = nullptr;      // maxit+2
  double* gmem = nullptr;      // backing store of gd
  ncs::GmresDev gd;
  ncs::GmresState* st_host = nullptr;  // pinned copy of *gd.st, read after each step
  // one captured Arnoldi step (product + orthogonalisation + state copy) per precision, and
  // (slot 4) for the inner FP32 products of the mixed solve
  static constexpr int kGraphSlots = 5;
  cudaGraphExec_t step_graph[kGraphSlots] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  long long step_graph_kernels[kGraphSlots] = {0, 0, 0, 0, 0};
  ncs_tuning tune{16, 4, 4, 16, 0.1, 0, 0};  // tree product launch configuration (ncs_tune)
  // one-patch data of the near-patch quadrature (ncs_eval), uploaded on first use
  bool near_ready = false;
  double* near_d = nullptr;
  int* near_i = nullptr;
  ncs::NearEvalArgs near_args{};
  bool graphs_off = false;      // capture failed once: steps are launched directly
  std::string graph_note;       // why
  double solve_stats[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // see ncs_solve_stats
};
