// The C-ABI of include/hsweep.h: argument checks, handle lifetime, factor-store
// layout, host<->device copies of single layers, and the rules that let the apply be
// captured into a CUDA graph (no allocation during a capture; buffers a captured graph
// may point into are kept until the handle is freed).
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include "handle.h"

// Test hook: HSWEEP_FAIL_ALLOC_AT=k (or "k:label") makes the k-th device allocation
// counted from the moment the variable took its current value fail with HSWEEP_ERR_OOM;
// a new value (another k or label) restarts the count, so one process can fail every
// allocation of a sequence in turn.
static bool alloc_hook_fires() {
  static std::mutex mu;
  static std::string last;
  static long long counter = 0, fail_at = -1;
  std::lock_guard<std::mutex> lock(mu);
  const char* e = getenv("HSWEEP_FAIL_ALLOC_AT");
  const std::string cur = e ? e : "";
  if (cur != last) {
    last = cur;
    counter = 0;
    fail_at = cur.empty() ? -1 : atoll(cur.c_str());
  }
  ++counter;
  return fail_at > 0 && counter == fail_at;
}

int hsw_alloc(hsweep_s* h, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (alloc_hook_fires()) return HSWEEP_ERR_OOM;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? HSWEEP_ERR_OOM : HSWEEP_ERR_CUDA;
  }
  h->allocs.push_back(*p);
  return HSWEEP_OK;
}

void hsw_release(hsweep_s* h, void* p) {
  if (!p) return;
  for (size_t i = 0; i < h->allocs.size(); ++i)
    if (h->allocs[i] == p) {
      cudaFree(p);
      h->allocs[i] = h->allocs.back();
      h->allocs.pop_back();
      return;
    }
}

bool hsw_capturing(hsweep_s* h) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(h->stream, &st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return st != cudaStreamCaptureStatusNone;
}

int hsw_regrow(hsweep_s* h, void** p, size_t bytes) {
  if (hsw_capturing(h)) return HSWEEP_ERR_ARG;
  if (!h->graph_held) hsw_release(h, *p);
  *p = nullptr;
  return hsw_alloc(h, p, bytes);
}

extern "C" int hsweep_default_opts(hsweep_opts* o) {
  if (!o) return HSWEEP_ERR_ARG;
  o->leaf = 8;
  o->r_max = 48;
  o->precision = HSWEEP_MIXED;
  o->pml_C = 6.283185307179586476925286766559;
  o->pml_form = 0;
  o->gmres_max_it = 60;
  o->refine_max = 8;
  o->team = 0;
  o->groups = 0;
  o->sweep_kernel = 0;
  o->sweep_tc = 0;
  o->sweep_dir = 1;
  o->pml_sides = 15;
  o->strong_rank = 0;
  o->rsvd_seed = 0;
  o->team_threads = 0;
  o->core_kernel = 0;
  o->krylov_lowp = 0;
  return HSWEEP_OK;
}

static void destroy(hsweep_s* h) {
  if (!h) return;
  hsw_setup_free(h);
  hsw_strong_free(h);
  hsw_spack_free(h);
  hsw_krylov_free(h);
  for (auto& pr : h->ev_sweep) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
  for (cudaEvent_t e : h->ev_free) cudaEventDestroy(e);
  h->ev_sweep.clear();
  h->ev_free.clear();
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  delete h;
}

extern "C" void hsweep_free(hsweep_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  destroy(h);
}

static int create_impl(const double* c_dev, double omega, int n, int pml_width, double eps_H,
                       const hsweep_opts* opt_in, void* stream, hsweep_t* out) {
  if (!out) return HSWEEP_ERR_ARG;
  *out = nullptr;
  hsweep_opts opt;
  hsweep_default_opts(&opt);
  if (opt_in) opt = *opt_in;
  if (!c_dev || !(omega > 0) || n < 3 || n > 32767 || pml_width < 0 || 2 * pml_width >= n ||
      !(eps_H >= 0) || opt.leaf < 2 || opt.leaf > 8 || opt.r_max < 1 || opt.r_max > 56 ||
      (opt.precision != HSWEEP_FP64 && opt.precision != HSWEEP_MIXED) || !(opt.pml_C >= 0) ||
      (opt.pml_form != 0 && opt.pml_form != 1) || opt.gmres_max_it < 1 || opt.gmres_max_it > 500 ||
      opt.refine_max < 1 || opt.team < 0 || opt.groups < 0 || opt.sweep_kernel < 0 || opt.sweep_kernel > 2 ||
      opt.sweep_tc < 0 || opt.sweep_tc > 2 ||
      (opt.sweep_dir != 1 && opt.sweep_dir != -1) || opt.pml_sides < 0 || opt.pml_sides > 15 ||
      opt.strong_rank < 0 || opt.strong_rank > 8 || opt.krylov_lowp < 0 || opt.krylov_lowp > 1 ||
      (opt.team_threads != 0 && opt.team_threads != 256 && opt.team_threads != 512) ||
      opt.core_kernel < 0 || opt.core_kernel > 2)
    return HSWEEP_ERR_ARG;
  hsweep_s* h = new (std::nothrow) hsweep_s();
  if (!h) return HSWEEP_ERR_OOM;
  h->n = n;
  h->N = n * n;
  h->pml_width = pml_width;
  h->omega = omega;
  h->h = 1.0 / (n + 1);
  h->eps_H = eps_H;
  h->opt = opt;
  h->stream = (cudaStream_t)stream;
  h->tree.build(n, opt.leaf);
  h->L = h->tree.L;
  h->leaf = opt.leaf;
  h->nnodes = h->tree.nnodes;
  h->nleaves = h->tree.nleaves;
  h->r_max = opt.r_max;
  h->strong_R = opt.strong_rank;
  if (h->strong_R > 0) {
    // the expanded strong form needs this rank at depth 1
    const int need = hsw_strong_expansion_rank(h->strong_R, h->L, h->leaf);
    if (need > 56) { delete h; return HSWEEP_ERR_ARG; }
    h->r_max = std::max(h->r_max, need);
  }
  h->prec = opt.precision;
  h->dir = opt.sweep_dir;
  int rc = HSWEEP_OK;
#define TRY(x) do { rc = (x); if (rc != HSWEEP_OK) { destroy(h); return rc; } } while (0)
#define TRYC(x) do { if ((x) != cudaSuccess) { cudaGetLastError(); destroy(h); return HSWEEP_ERR_CUDA; } } while (0)
  TRYC(cudaGetDevice(&h->device));
  TRYC(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
  hsw_noalloc_bind(h);

  // factor-store layout (identical for every layer)
  h->off.assign(h->nnodes, 0);
  h->leaf_entries = (long long)h->nleaves * h->leaf * h->leaf;
  long long o = h->leaf_entries;
  for (int v = 2; v < h->nnodes; ++v) {
    h->off[v] = o;
    o += (long long)h->tree.sz[v] * h->r_max;
  }
  o = (o + 31) & ~31LL;   // keep every layer 256-byte aligned
  h->layer_stride = o;
  // packed copy: worst-case record of every leaf (all ranks at r_max), layers 256-byte aligned
  {
    const long long rs = h->r_max | 1;
    const long long rec = (long long)h->leaf * h->leaf + (long long)h->L * h->leaf * rs + 1;
    h->pack_stride = ((long long)h->nleaves * rec + 31) & ~31LL;
  }

  const size_t N = (size_t)h->N;
  TRY(hsw_alloc(h, (void**)&h->d_lo, h->nnodes * sizeof(int)));
  TRY(hsw_alloc(h, (void**)&h->d_sz, h->nnodes * sizeof(int)));
  TRY(hsw_alloc(h, (void**)&h->d_off, h->nnodes * sizeof(long long)));
  TRY(hsw_alloc(h, &h->d_fac, (size_t)n * h->layer_stride * h->fac_elem()));
  TRY(hsw_alloc(h, (void**)&h->d_rank, (size_t)n * h->nnodes * sizeof(int)));
  TRY(hsw_alloc(h, (void**)&h->d_c, N * sizeof(double)));
  TRY(hsw_alloc(h, (void**)&h->d_diag, N * sizeof(c128)));
  TRY(hsw_alloc(h, (void**)&h->d_east, (size_t)n * (n + 1) * sizeof(c128)));
  TRY(hsw_alloc(h, (void**)&h->d_north, (size_t)(n + 1) * n * sizeof(c128)));
  TRY(hsw_alloc(h, (void**)&h->d_s1s2, N * sizeof(c128)));
  TRY(hsw_alloc(h, &h->d_pack, (size_t)n * h->pack_stride * h->fac_elem()));
  TRY(hsw_alloc(h, (void**)&h->d_recoff, (size_t)n * (h->nleaves + 1) * sizeof(long long)));
  TRY(hsw_alloc(h, (void**)&h->d_status, 2 * sizeof(int)));
  TRY(hsw_alloc(h, (void**)&h->d_bar, 2 * sizeof(unsigned)));
  TRYC(cudaMemcpyAsync(h->d_lo, h->tree.lo.data(), h->nnodes * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  TRYC(cudaMemcpyAsync(h->d_sz, h->tree.sz.data(), h->nnodes * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  TRYC(cudaMemcpyAsync(h->d_off, h->off.data(), h->nnodes * sizeof(long long), cudaMemcpyHostToDevice, h->stream));
  TRYC(cudaMemsetAsync(h->d_fac, 0, (size_t)n * h->layer_stride * h->fac_elem(), h->stream));
  TRYC(cudaMemsetAsync(h->d_rank, 0, (size_t)n * h->nnodes * sizeof(int), h->stream));
  TRYC(cudaMemsetAsync(h->d_recoff, 0, (size_t)n * (h->nleaves + 1) * sizeof(long long), h->stream));
  TRYC(cudaMemsetAsync(h->d_status, 0, 2 * sizeof(int), h->stream));
  TRYC(cudaMemsetAsync(h->d_bar, 0, 2 * sizeof(unsigned), h->stream));
  if (h->dir < 0) TRY(hsw_flip_real(h, c_dev, h->d_c));   // the reflected problem
  else TRYC(cudaMemcpyAsync(h->d_c, c_dev, N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  // the velocity must be finite and positive
  {
    std::vector<double> hc(N);
    TRYC(cudaMemcpyAsync(hc.data(), c_dev, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    TRYC(cudaStreamSynchronize(h->stream));
    for (size_t i = 0; i < N; ++i)
      if (!(hc[i] > 0) || !std::isfinite(hc[i])) { destroy(h); return HSWEEP_ERR_ARG; }
  }
  {
    // the reflected problem of a downward sweep swaps the layers at x2 = 0 and x2 = 1
    int sides = opt.pml_sides;
    if (h->dir < 0) sides = (sides & 3) | ((sides & 4) << 1) | ((sides & 8) >> 1);
    TRY(hsw_assemble(h, opt.pml_C, opt.pml_form, sides, h->d_diag, h->d_east, h->d_north, h->d_s1s2));
    h->d_diag_m = h->d_diag;
    h->d_east_m = h->d_east;
    h->d_north_m = h->d_north;
    if (pml_width > 0 && (sides & 4) == 0) {
      // The sweep starts at a Dirichlet side (x2 = 0 of the stored problem).  Without
      // absorption there, the Schur-complement recursion S_m = A_mm - A T_{m-1} A amplifies
      // truncation and rounding errors from layer to layer (the perturbation of T_m is
      // about a^2 T_m dT_{m-1} T_m, with a^2 ~ 1/h^4 and |T_m| no longer small), and the
      // factorised T~_m drift from the exact ones within a few wavelengths.  The
      // factorisation is therefore built for the operator with an absorbing layer of the
      // same width and profile on that side; GMRES still solves the true A u = f.
      TRY(hsw_alloc(h, (void**)&h->d_diag_m, N * sizeof(c128)));
      TRY(hsw_alloc(h, (void**)&h->d_east_m, (size_t)n * (n + 1) * sizeof(c128)));
      TRY(hsw_alloc(h, (void**)&h->d_north_m, (size_t)(n + 1) * n * sizeof(c128)));
      TRY(hsw_assemble(h, opt.pml_C, opt.pml_form, sides | 4, h->d_diag_m, h->d_east_m, h->d_north_m, nullptr));
      h->start_absorber = true;
    }
  }
  TRYC(cudaStreamSynchronize(h->stream));
#undef TRY
#undef TRYC
  *out = h;
  return HSWEEP_OK;
}

extern "C" int hsweep_create(const double* c_dev, double omega, int n, int pml_width, double eps_H,
                             const hsweep_opts* opt, void* stream, hsweep_t* out) {
  return create_impl(c_dev, omega, n, pml_width, eps_H, opt, stream, out);
}

extern "C" int hsweep_setup(const double* c_dev, double omega, int n, int pml_width, double eps_H,
                            const hsweep_opts* opt, void* stream, hsweep_t* out) {
  if (!out) return HSWEEP_ERR_ARG;
  NvtxRange range("hsweep_setup");
  hsweep_t h = nullptr;
  int rc = create_impl(c_dev, omega, n, pml_width, eps_H, opt, stream, &h);
  if (rc != HSWEEP_OK) return rc;
  rc = hsw_factor(h);
  if (rc == HSWEEP_OK) {
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = HSWEEP_ERR_CUDA;
  }
  hsw_setup_free(h);   // the setup workspace is not needed once the factors are stored
  if (rc == HSWEEP_OK) rc = hsw_pack(h, 0, h->n);
  if (rc == HSWEEP_OK) {
    int st[2] = {0, -1};
    if (cudaMemcpy(st, h->d_status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) rc = HSWEEP_ERR_CUDA;
    else if (st[0] != 0) rc = st[0];
  }
  if (rc != HSWEEP_OK) {
    hsweep_free(h);
    return rc;
  }
  *out = h;
  return HSWEEP_OK;
}

extern "C" int hsweep_apply(hsweep_t h, const hsw_c128* r, hsw_c128* z, int nrhs) {
  if (!h || nrhs < 0 || (nrhs > 0 && (!r || !z))) return HSWEEP_ERR_ARG;
  NvtxRange range("hsweep_apply");
  const char* rb = (const char*)r;
  const char* zb = (const char*)z;
  size_t bytes = (size_t)nrhs * h->N * sizeof(hsw_c128);
  if (nrhs > 0 && rb < zb + bytes && zb < rb + bytes) return HSWEEP_ERR_ARG;
  if (nrhs > 0 && hsw_capturing(h)) {
    // stream capture: upward handles only; no timing events inside a graph
    if (h->dir < 0) return HSWEEP_ERR_ARG;
    h->graph_held = true;
    const bool prof = h->prof;
    h->prof = false;
    const int rc = hsw_apply(h, reinterpret_cast<const c128*>(r), reinterpret_cast<c128*>(z), nrhs);
    h->prof = prof;
    return rc;
  }
  if (h->dir > 0 || nrhs == 0) return hsw_apply(h, reinterpret_cast<const c128*>(r), reinterpret_cast<c128*>(z), nrhs);
  // downward sweep: z = P M' P r with M' the upward sweep of the reflected problem
  int rc = hsw_flip_reserve(h, 2 * bytes);
  if (rc) return rc;
  c128* a = static_cast<c128*>(h->d_flip);
  c128* b = a + (size_t)nrhs * h->N;
  if ((rc = hsw_flip_c128(h, reinterpret_cast<const c128*>(r), a, nrhs))) return rc;
  if ((rc = hsw_apply(h, a, b, nrhs))) return rc;
  return hsw_flip_c128(h, b, reinterpret_cast<c128*>(z), nrhs);
}

extern "C" int hsweep_matvec(hsweep_t h, const hsw_c128* x, hsw_c128* y, int nrhs) {
  if (!h || nrhs < 0 || (nrhs > 0 && (!x || !y))) return HSWEEP_ERR_ARG;
  const char* xb = (const char*)x;
  const char* yb = (const char*)y;
  size_t bytes = (size_t)nrhs * h->N * sizeof(hsw_c128);
  if (nrhs > 0 && xb < yb + bytes && yb < xb + bytes) return HSWEEP_ERR_ARG;
  if (h->dir > 0 || nrhs == 0) return hsw_matvec(h, reinterpret_cast<const c128*>(x), reinterpret_cast<c128*>(y), nrhs);
  int rc = hsw_flip_reserve(h, 2 * bytes);
  if (rc) return rc;
  c128* a = static_cast<c128*>(h->d_flip);
  c128* b = a + (size_t)nrhs * h->N;
  if ((rc = hsw_flip_c128(h, reinterpret_cast<const c128*>(x), a, nrhs))) return rc;
  if ((rc = hsw_matvec(h, a, b, nrhs))) return rc;
  return hsw_flip_c128(h, b, reinterpret_cast<c128*>(y), nrhs);
}

extern "C" int hsweep_solve(hsweep_t h, const hsw_c128* f, hsw_c128* u, int nrhs, double tol,
                            int* iters_out, double* relres_out) {
  if (!h || nrhs < 0 || (nrhs > 0 && (!f || !u)) || !(tol > 0) || tol >= 1) return HSWEEP_ERR_ARG;
  if (nrhs == 0) return HSWEEP_OK;
  NvtxRange range("hsweep_solve");
  if (h->dir > 0)
    return hsw_solve(h, reinterpret_cast<const c128*>(f), reinterpret_cast<c128*>(u), nrhs, tol,
                     iters_out, relres_out);
  const size_t bytes = (size_t)nrhs * h->N * sizeof(c128);
  int rc = hsw_flip_reserve(h, 2 * bytes);
  if (rc) return rc;
  c128* a = static_cast<c128*>(h->d_flip);
  c128* b = a + (size_t)nrhs * h->N;
  if ((rc = hsw_flip_c128(h, reinterpret_cast<const c128*>(f), a, nrhs))) return rc;
  if ((rc = hsw_flip_c128(h, reinterpret_cast<const c128*>(u), b, nrhs))) return rc;
  const int rs = hsw_solve(h, a, b, nrhs, tol, iters_out, relres_out);
  if (rs != HSWEEP_OK && rs != HSWEEP_ERR_NOT_CONVERGED) return rs;
  if ((rc = hsw_flip_c128(h, b, reinterpret_cast<c128*>(u), nrhs))) return rc;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return HSWEEP_ERR_CUDA;
  return rs;
}

extern "C" int hsweep_grad(hsweep_t h, const hsw_c128* f, int nsrc, const int* rec_idx, int nrec,
                           const hsw_c128* d, double* grad, double* misfit_out, double tol) {
  if (!h || nsrc < 1 || nrec < 1 || !f || !rec_idx || !d || !grad || !(tol > 0) || tol >= 1)
    return HSWEEP_ERR_ARG;
  NvtxRange range("hsweep_grad");
  if (h->dir > 0)
    return hsw_grad(h, reinterpret_cast<const c128*>(f), nsrc, rec_idx, nrec,
                    reinterpret_cast<const c128*>(d), grad, misfit_out, tol);
  // the reflected problem: sources and receiver nodes through P, the gradient back
  const size_t fb = (size_t)nsrc * h->N * sizeof(c128);
  const size_t rb = ((size_t)nrec * sizeof(int) + 255) / 256 * 256;
  int rc = hsw_flip_reserve(h, fb + rb + (size_t)h->N * sizeof(double));
  if (rc) return rc;
  c128* fa = static_cast<c128*>(h->d_flip);
  int* ra = reinterpret_cast<int*>(static_cast<unsigned char*>(h->d_flip) + fb);
  double* ga = reinterpret_cast<double*>(static_cast<unsigned char*>(h->d_flip) + fb + rb);
  if ((rc = hsw_flip_c128(h, reinterpret_cast<const c128*>(f), fa, nsrc))) return rc;
  if ((rc = hsw_flip_index(h, rec_idx, ra, nrec))) return rc;
  if ((rc = hsw_grad(h, fa, nsrc, ra, nrec, reinterpret_cast<const c128*>(d), ga, misfit_out, tol))) return rc;
  if ((rc = hsw_flip_real(h, ga, grad))) return rc;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return HSWEEP_ERR_CUDA;
  return HSWEEP_OK;
}

extern "C" int hsweep_boundary_rhs(hsweep_t h, int side, const hsw_c128* b, hsw_c128* f, int nrhs) {
  if (!h || side < 0 || side > 3 || nrhs < 0 || (nrhs > 0 && (!b || !f))) return HSWEEP_ERR_ARG;
  return hsw_boundary_rhs(h, side, reinterpret_cast<const c128*>(b), reinterpret_cast<c128*>(f), nrhs);
}

extern "C" int hsweep_status(hsweep_t h, int* layer_out) {
  if (!h) return HSWEEP_ERR_ARG;
  int st[2] = {0, -1};
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return HSWEEP_ERR_CUDA;
  if (cudaMemcpy(st, h->d_status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return HSWEEP_ERR_CUDA;
  if (layer_out) *layer_out = st[0] ? st[1] : -1;
  return st[0];
}

extern "C" int hsweep_info(hsweep_t h, long long* out8) {
  if (!h || !out8) return HSWEEP_ERR_ARG;
  std::vector<int> rk((size_t)h->n * h->nnodes);
  HSW_CUDA(cudaStreamSynchronize(h->stream));
  HSW_CUDA(cudaMemcpy(rk.data(), h->d_rank, rk.size() * sizeof(int), cudaMemcpyDeviceToHost));
  long long entries = 0;
  for (int m = 0; m < h->n; ++m) {
    entries += h->leaf_entries;
    for (int v = 2; v < h->nnodes; ++v) entries += (long long)h->tree.sz[v] * rk[(size_t)m * h->nnodes + v];
  }
  out8[0] = h->n; out8[1] = h->L; out8[2] = h->leaf; out8[3] = h->r_max;
  out8[4] = h->prec; out8[5] = h->nleaves; out8[6] = entries; out8[7] = (long long)h->fac_elem();
  return HSWEEP_OK;
}

extern "C" int hsweep_layer_ranks(hsweep_t h, int m, int* ranks_out) {
  if (!h || m < 0 || m >= h->n || !ranks_out) return HSWEEP_ERR_ARG;
  HSW_CUDA(cudaStreamSynchronize(h->stream));
  HSW_CUDA(cudaMemcpy(ranks_out, h->d_rank + (size_t)m * h->nnodes, h->nnodes * sizeof(int),
                      cudaMemcpyDeviceToHost));
  return HSWEEP_OK;
}

// Host packing between the layer layout on the device and the complex128 host layout.
static size_t layer_host_entries(const hsweep_s* h) {
  return (size_t)h->layer_stride;
}

extern "C" int hsweep_export_layer(hsweep_t h, int m, hsw_c128* leaves, hsw_c128* factors, int* ranks) {
  if (!h || m < 0 || m >= h->n || !leaves || !factors || !ranks) return HSWEEP_ERR_ARG;
  size_t ne = layer_host_entries(h);
  std::vector<unsigned char> buf(ne * h->fac_elem());
  HSW_CUDA(cudaStreamSynchronize(h->stream));
  HSW_CUDA(cudaMemcpy(buf.data(), (const char*)h->d_fac + (size_t)m * h->layer_stride * h->fac_elem(),
                      buf.size(), cudaMemcpyDeviceToHost));
  HSW_CUDA(cudaMemcpy(ranks, h->d_rank + (size_t)m * h->nnodes, h->nnodes * sizeof(int), cudaMemcpyDeviceToHost));
  auto get = [&](size_t i) -> hsw_c128 {
    if (h->prec == HSWEEP_FP64) { const c128* p = (const c128*)buf.data(); return {p[i].re, p[i].im}; }
    const c64* p = (const c64*)buf.data();
    return {(double)p[i].re, (double)p[i].im};
  };
  for (long long i = 0; i < h->leaf_entries; ++i) leaves[i] = get(i);
  size_t fo = 0;
  for (int v = 2; v < h->nnodes; ++v) {
    size_t cnt = (size_t)h->tree.sz[v] * h->r_max;
    for (size_t i = 0; i < cnt; ++i) factors[fo + i] = get(h->off[v] + i);
    fo += cnt;
  }
  return HSWEEP_OK;
}

extern "C" int hsweep_import_layer(hsweep_t h, int m, const hsw_c128* leaves, const hsw_c128* factors,
                                   const int* ranks) {
  if (!h || m < 0 || m >= h->n || !leaves || !factors || !ranks) return HSWEEP_ERR_ARG;
  for (int v = 2; v < h->nnodes; ++v)
    if (ranks[v] < 0 || ranks[v] > h->r_max || ranks[v] != ranks[v ^ 1]) return HSWEEP_ERR_ARG;
  size_t ne = layer_host_entries(h);
  std::vector<unsigned char> buf(ne * h->fac_elem(), 0);
  auto put = [&](size_t i, hsw_c128 v) {
    if (h->prec == HSWEEP_FP64) { ((c128*)buf.data())[i] = c128(v.re, v.im); }
    else { ((c64*)buf.data())[i] = c64((float)v.re, (float)v.im); }
  };
  for (long long i = 0; i < h->leaf_entries; ++i) put(i, leaves[i]);
  size_t fo = 0;
  for (int v = 2; v < h->nnodes; ++v) {
    size_t cnt = (size_t)h->tree.sz[v] * h->r_max;
    for (size_t i = 0; i < cnt; ++i) put(h->off[v] + i, factors[fo + i]);
    fo += cnt;
  }
  std::vector<int> rk(ranks, ranks + h->nnodes);
  rk[0] = rk[1] = 0;
  HSW_CUDA(cudaStreamSynchronize(h->stream));
  HSW_CUDA(cudaMemcpy((char*)h->d_fac + (size_t)m * h->layer_stride * h->fac_elem(), buf.data(), buf.size(),
                      cudaMemcpyHostToDevice));
  HSW_CUDA(cudaMemcpy(h->d_rank + (size_t)m * h->nnodes, rk.data(), h->nnodes * sizeof(int), cudaMemcpyHostToDevice));
  h->spack_valid = false;   // the strong sweep's records no longer describe the factors
  return hsw_pack(h, m, m + 1);
}

extern "C" int hsweep_set_stream(hsweep_t h, void* stream) {
  if (!h) return HSWEEP_ERR_ARG;
  h->stream = (cudaStream_t)stream;
  return HSWEEP_OK;
}

extern "C" int hsweep_profile(hsweep_t h, int enable) {
  if (!h) return HSWEEP_ERR_ARG;
  h->prof = enable != 0;
  return HSWEEP_OK;
}

extern "C" int hsweep_stats(hsweep_t h, int reset, long long* launches, long long* sweep_launches,
                            double* sweep_ms) {
  if (!h) return HSWEEP_ERR_ARG;
  HSW_CUDA(cudaStreamSynchronize(h->stream));
  double ms = 0;
  for (auto& pr : h->ev_sweep) {
    float t = 0;
    HSW_CUDA(cudaEventElapsedTime(&t, pr.first, pr.second));
    ms += t;
  }
  if (launches) *launches = h->nlaunch;
  if (sweep_launches) *sweep_launches = (long long)h->ev_sweep.size();
  if (sweep_ms) *sweep_ms = ms;
  if (reset) {
    h->nlaunch = 0;
    for (auto& pr : h->ev_sweep) { h->ev_free.push_back(pr.first); h->ev_free.push_back(pr.second); }
    h->ev_sweep.clear();
  }
  return HSWEEP_OK;
}

extern "C" int hsweep_setup_tuning(hsweep_t h, double* out6) {
  if (!h || !out6) return HSWEEP_ERR_ARG;
  for (int k = 0; k < 2; ++k) {
    out6[k] = h->core_mode[k];
    out6[2 + 2 * k] = h->core_ms[k][0];
    out6[3 + 2 * k] = h->core_ms[k][1];
  }
  return HSWEEP_OK;
}

extern "C" int hsweep_sweep_plan(hsweep_t h, int nrhs, long long* out8) {
  if (!h || !out8 || nrhs < 1) return HSWEEP_ERR_ARG;
  if (h->opt.sweep_kernel == 0 && h->strong_R > 0 && hsw_strong_plan_sweep(h, nrhs, out8)) return HSWEEP_OK;
  if (h->opt.sweep_kernel != 1 && hsw_team_plan(h, nrhs, out8)) return HSWEEP_OK;
  for (int i = 0; i < 8; ++i) out8[i] = 0;
  return HSWEEP_OK;
}
