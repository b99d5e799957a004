// Internal state of an hsweep handle, shared by the translation units of the library.
#pragma once
#include <array>
#include <utility>
#include <vector>
#include <nvtx3/nvToolsExt.h>
#include "common.cuh"

// NVTX range over a phase of the method (setup, a setup layer, apply, solve, a GMRES step,
// gradient), visible on profiler timelines; a push and a pop cost nanoseconds without a tool
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Cluster tree of one layer (Section 2.3): heap-indexed nodes, root = 1, children of v
// are 2v and 2v+1; a node [lo, lo+sz) of size s splits into ceil(s/2) and floor(s/2)
// rows; all leaves sit at depth L, the smallest L with ceil(n / 2^L) <= leaf.
struct Tree {
  int n = 0, L = 0, leaf = 0, nnodes = 0, nleaves = 0;
  std::vector<int> lo, sz;
  void build(int n_, int leaf_) {
    n = n_; leaf = leaf_;
    L = 0;
    while ((n + (1 << L) - 1) / (1 << L) > leaf) ++L;
    nnodes = 1 << (L + 1);
    nleaves = 1 << L;
    lo.assign(nnodes, 0); sz.assign(nnodes, 0);
    lo[1] = 0; sz[1] = n;
    for (int v = 1; v < nnodes / 2; ++v) {
      int a = (sz[v] + 1) / 2;
      lo[2 * v] = lo[v]; sz[2 * v] = a;
      lo[2 * v + 1] = lo[v] + a; sz[2 * v + 1] = sz[v] - a;
    }
  }
  // largest node size at depth d
  int maxsz(int d) const { return (n + (1 << d) - 1) >> d; }
};

struct SetupWork;   // setup.cu
struct StrongWork;  // strong.cu
struct StrongPack;  // sweep_strong.cu
struct KrylovWork;  // krylov.cu

struct hsweep_s {
  int n = 0, N = 0, pml_width = 0;
  double omega = 0, h = 0, eps_H = 0;
  hsweep_opts opt{};
  Tree tree;
  int L = 0, leaf = 0, nnodes = 0, nleaves = 0, r_max = 0, prec = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0, device = 0;

  // factor store: layer m occupies [m * layer_stride, (m+1) * layer_stride) entries;
  // leaves first (nleaves * leaf * leaf), then F_v (sz[v] x r_max, column-major) at off[v].
  std::vector<long long> off;
  long long layer_stride = 0, leaf_entries = 0;
  int* d_lo = nullptr;
  int* d_sz = nullptr;
  long long* d_off = nullptr;
  void* d_fac = nullptr;   // c64 (HSWEEP_MIXED) or c128 (HSWEEP_FP64)
  int* d_rank = nullptr;   // [n][nnodes]

  // discretisation (complex128): diag [n][n], east [n][n+1], north [n+1][n], s1s2 [n][n]
  double* d_c = nullptr;
  c128* d_diag = nullptr;
  c128* d_east = nullptr;
  c128* d_north = nullptr;
  c128* d_s1s2 = nullptr;
  // the operator the sweeping factorisation is built for (setup and the apply's layer
  // couplings): the arrays above, except when the sweep starts at a side without a PML;
  // then its own arrays, assembled with an absorbing layer on that side (api.cu)
  c128* d_diag_m = nullptr;
  c128* d_east_m = nullptr;
  c128* d_north_m = nullptr;
  bool start_absorber = false;

  // Leaf-major packed copy of the factors, read by the sweep: for every layer and leaf
  // one contiguous record [leaf block | rows of the leaf in F_v for depths 1..L], so the
  // rows of any subtree form one contiguous byte range (see pack.cu).
  void* d_pack = nullptr;
  long long pack_stride = 0;             // entries per layer (worst-case capacity)
  long long* d_recoff = nullptr;         // [n][nleaves + 1] record offsets within a layer
  std::vector<long long> slab_bytes_max; // per slab depth dC: largest slab record in bytes
  // team-sweep launch plans already chosen: {nrhs, ok, dC, C, G, teams, smem, threads per
  // CTA}; cleared whenever the packed factors change
  std::vector<std::array<long long, 8>> team_plans;
  int rank_max = 0;
  std::vector<int> rank_max_depth;       // per depth d = 0..L: the largest rank over all layers
  bool pack_valid = false;

  int* d_status = nullptr;     // [2]
  unsigned* d_bar = nullptr;   // grid barrier words [2]

  // sweep workspace
  void* d_wcache = nullptr;    // [cap][N] in storage precision
  void* d_xch = nullptr;       // team exchange slots
  long long wcache_cap = 0, xch_cap = 0;

  // sweep direction: +1 upward from x2 = 0 (Algorithm 2.5), -1 downward (the handle holds
  // the reflected problem; direction.cu) with a scratch for the reflected vectors
  int dir = 1;
  void* d_flip = nullptr;
  size_t flip_cap = 0;

  SetupWork* sw = nullptr;
  KrylovWork* kw = nullptr;
  // strong admissibility (strong.cu): rank R of the well-separated blocks, 0 = weak
  int strong_R = 0;
  StrongWork* stw = nullptr;
  // the strongly admissible T~_m in their own format for the strong sweep (sweep_strong.cu),
  // written by the setup; an imported layer invalidates them
  StrongPack* spk = nullptr;
  bool spack_valid = false;

  std::vector<void*> allocs;   // every device allocation owned by the handle

  // setup autotuning of the recompression's core products (setup.cu): per kind of launch
  // (0: after a depth step, 1: once per layer) the kernel kept (-1 not tuned, 0 CUDA cores,
  // 1 tensor cores) and the two candidates' times in milliseconds
  int core_mode[2] = {-1, -1};
  float core_ms[2][2] = {{0, 0}, {0, 0}};

  // device address of the library's fixed scratch array for hsweep_apply_noalloc, looked
  // up on the handle's device when the handle is created (noalloc.cu); null if that failed
  void* noalloc_scratch = nullptr;

  // instrumentation: kernel launches made by this handle, and (when prof is set) a
  // pair of CUDA events around every sweep-kernel launch on the handle's stream
  long long nlaunch = 0;
  bool prof = false;
  // set once an apply was called while the handle's stream was being captured into a CUDA
  // graph: from then on, buffers that later calls outgrow stay allocated until hsweep_free,
  // because the graph's launches still point into them
  bool graph_held = false;
  std::vector<cudaEvent_t> ev_free;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_sweep;

  size_t fac_elem() const { return prec == HSWEEP_FP64 ? sizeof(c128) : sizeof(c64); }
};

// Device allocation owned by the handle; HSWEEP_ERR_OOM on failure.
int hsw_alloc(hsweep_s* h, void** p, size_t bytes);
void hsw_release(hsweep_s* h, void* p);
// true while the handle's stream is being captured into a CUDA graph
bool hsw_capturing(hsweep_s* h);
// *p replaced by a new buffer of `bytes` (contents not kept) for the apply's scratch (the w
// cache, the exchange slots, the reflected vectors): HSWEEP_ERR_ARG during a capture (size the
// buffers with one call outside it); the old buffer is released unless graph_held is set
int hsw_regrow(hsweep_s* h, void** p, size_t bytes);

// assemble.cu: the operator with PMLs on the sides in pml_sides into diag/east/north
// (and s1s2 unless null)
int hsw_assemble(hsweep_s* h, double pml_C, int pml_form, int pml_sides, c128* diag, c128* east, c128* north,
                 c128* s1s2);
// Dirichlet data b on one side as a forcing term on the adjacent layer (Section 2.5)
int hsw_boundary_rhs(hsweep_s* h, int side, const c128* b, c128* f, int nrhs);
int hsw_matvec(hsweep_s* h, const c128* x, c128* y, int nrhs);
// r = f - A u (FP64), one pass
int hsw_residual(hsweep_s* h, const c128* f, const c128* u, c128* r, int nrhs);
// the same product with FP32 arithmetic (lowp) on the FP64 vectors
int hsw_matvec_prec(hsweep_s* h, const c128* x, c128* y, int nrhs, bool lowp);
// noalloc.cu: look up the fixed scratch array on the current (the handle's) device
void hsw_noalloc_bind(hsweep_s* h);
// apply.cu
int hsw_apply(hsweep_s* h, const c128* r, c128* z, int nrhs);
size_t hsw_apply_scratch_bytes(hsweep_s* h, int nrhs);
int hsw_apply_scratch(hsweep_s* h, const c128* r, c128* z, int nrhs, void* scratch, size_t bytes);
// pack.cu
int hsw_pack(hsweep_s* h, int m0, int m1);
// sweep_team.cu
int hsw_apply_team(hsweep_s* h, const c128* r, c128* z, int nrhs, bool* used, void* scratch = nullptr,
                   size_t scratch_bytes = 0);
size_t hsw_apply_team_scratch_bytes(hsweep_s* h, int nrhs);
int hsw_team_plan(hsweep_s* h, int nrhs, long long* out8);   // 1 if the team kernel would run
// direction.cu: reversal of the layer order (x2 -> 1 - x2)
int hsw_flip_reserve(hsweep_s* h, size_t bytes);
int hsw_flip_c128(hsweep_s* h, const c128* in, c128* out, int nvec);
int hsw_flip_real(hsweep_s* h, const double* in, double* out);
int hsw_flip_index(hsweep_s* h, const int* in, int* out, int cnt);
// strong.cu: rank-R projection of the weak T~_m onto the strongly admissible partition,
// written back into the factor buffers G_F2 (ranks into G_rank)
int hsw_strong_project(hsweep_s* h, int m, const void* G_F, int* G_rank, void* G_F2, const long long* d_gfo,
                       long long gf_entries);
int hsw_strong_expansion_rank(int R, int L, int leaf);
void hsw_strong_free(hsweep_s* h);
// sweep_strong.cu: records of layer m from the expanded strongly admissible factors (setup
// layout), the apply on them, its scratch and plan
int hsw_spack_layer(hsweep_s* h, int m, const void* G_F, const void* G_leaf, const long long* d_gfo);
void hsw_spack_free(hsweep_s* h);
int hsw_apply_strong(hsweep_s* h, const c128* r, c128* z, int nrhs, bool* used, void* scratch = nullptr,
                     size_t scratch_bytes = 0);
size_t hsw_apply_strong_scratch_bytes(hsweep_s* h, int nrhs);
int hsw_strong_plan_sweep(hsweep_s* h, int nrhs, long long* out8);   // 1 if the strong sweep would run
__host__ __device__ void hsw_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
// setup.cu
int hsw_factor(hsweep_s* h);
void hsw_setup_free(hsweep_s* h);
// krylov.cu
int hsw_solve(hsweep_s* h, const c128* f, c128* u, int nrhs, double tol, int* iters, double* relres);
void hsw_krylov_free(hsweep_s* h);
// grad.cu
int hsw_grad(hsweep_s* h, const c128* f, int nsrc, const int* rec, int nrec, const c128* d,
             double* grad, double* misfit, double tol);
