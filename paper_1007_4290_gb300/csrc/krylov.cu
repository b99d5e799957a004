// GMRES on the left-preconditioned system M A u = M f (Section 2.4), batched over
// right-hand sides, with Arnoldi by classical Gram-Schmidt (a second pass where the
// first lost more than half of a vector's squared norm, except at the first step of an
// inner solve, where the loss of orthogonality is local and a tighter test applies), Givens
// rotations on the host, and an outer loop on the FP64 residual:
//     r = f - A u,  z = M r,  stop when ||z|| <= tol ||M f||,
//     otherwise GMRES on M A d = z (x0 = 0) and u += d.
// In HSWEEP_FP64 a converged inner solve ends the loop (its residual estimate is the
// FP64 one); in HSWEEP_MIXED, where M runs in complex64, every outer step re-checks
// the FP64 residual (iterative refinement).  The inner GMRES (Arnoldi by Gram-Schmidt,
// norms, scalings, the product with A) computes in FP64 in both modes.  The option
// krylov_lowp moves it to FP32 arithmetic on the FP64-stored vectors in HSWEEP_MIXED
// (the FP64 units of this GPU run at about 1/60 of the FP32 rate): per-thread products
// and partial sums in FP32, block and global sums in FP64.  In HSWEEP_MIXED the inner
// target is a relative 4e-6 at most in either arithmetic (the complex64 sweeps make M A
// accurate to a few 1e-7 only); the outer refinement reaches the tolerance, and its last
// step is accepted on the inner estimate once the sweep's rounding cannot matter (see
// kSweepNoise).  The residual f - A u, the update u += d and the reported residuals stay
// FP64 in every case.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include "handle.h"

namespace {

constexpr int kRedBlocks = 304;   // 2 x 152 SMs of partial sums per vector

constexpr int kDotChunk = 4;      // basis vectors per pass over w

// Bound on the relative departure of the complex64 sweep from a linear map,
// ||M(x + y) - M x - M y|| <= kSweepNoise (||M x|| + ||M y||) (measured well below it by
// the GPU tests of the mixed apply)
constexpr double kSweepNoise = 1e-5;

// partial[(s * nt + i) * B + b] = sum over block b's chunk of conj(V_i[s]) . w[s] for
// i < nv, and for i = nv (when nt = nv + 1) the squared norm of w[s]; w is read once per
// kDotChunk outputs; T = the per-thread arithmetic type
template <typename T>
__global__ void dots_kernel(const c128* const* __restrict__ V, int nv, int nt, const c128* __restrict__ w, long long N,
                            c128* __restrict__ partial) {
  const int s = blockIdx.y, B = gridDim.x;
  const long long chunk = (N + B - 1) / B;
  const long long beg = blockIdx.x * chunk, end = min(N, beg + chunk);
  __shared__ c128 red[kDotChunk][32];
  const c128* ws = w + s * N;
  for (int i0 = 0; i0 < nt; i0 += kDotChunk) {
    const int nc = min(kDotChunk, nt - i0);
    const c128* vs[kDotChunk];
#pragma unroll
    for (int i = 0; i < kDotChunk; ++i) {
      const int ii = i0 + (i < nc ? i : 0);
      vs[i] = ii < nv ? V[ii] + s * N : ws;
    }
    Cx<T> acct[kDotChunk];
#pragma unroll
    for (int i = 0; i < kDotChunk; ++i) acct[i] = Cx<T>(0, 0);
    for (long long p = beg + threadIdx.x; p < end; p += blockDim.x) {
      const Cx<T> wp = cvt<T>(ws[p]);
#pragma unroll
      for (int i = 0; i < kDotChunk; ++i) {
        if (i0 + i < nv) {
          if (i < nc) cfma_conj(acct[i], cvt<T>(vs[i][p]), wp);
        } else if (i < nc) {
          acct[i].re += abs2(wp);      // the squared norm: two multiply-adds, not four
        }
      }
    }
    c128 acc[kDotChunk];
#pragma unroll
    for (int i = 0; i < kDotChunk; ++i) {
      acc[i] = cvt<double>(acct[i]);
      for (int o = 16; o > 0; o >>= 1) acc[i] += shfl_xor(acc[i], o);
      if ((threadIdx.x & 31) == 0) red[i][threadIdx.x >> 5] = acc[i];
    }
    __syncthreads();
    if (threadIdx.x < nc) {
      c128 t(0, 0);
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[threadIdx.x][k];
      partial[((long long)s * nt + i0 + threadIdx.x) * B + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// partial[s * B + b] = sum over block b's chunk of |x[s]|^2 (as the real part)
template <typename T>
__global__ void sqnorm_kernel(const c128* __restrict__ x, long long N, c128* __restrict__ partial) {
  const int s = blockIdx.y, B = gridDim.x;
  const long long chunk = (N + B - 1) / B;
  const long long beg = blockIdx.x * chunk, end = min(N, beg + chunk);
  __shared__ double red[32];
  const c128* xs = x + s * N;
  T acct = T(0);
  for (long long p = beg + threadIdx.x; p < end; p += blockDim.x) acct += abs2(cvt<T>(xs[p]));
  double acc = acct;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    partial[(long long)s * B + blockIdx.x] = c128(t, 0.0);
  }
}

__global__ void reduce_partials(const c128* __restrict__ partial, int B, c128* __restrict__ out) {
  const int idx = blockIdx.x;
  __shared__ c128 red[32];
  c128 acc(0, 0);
  for (int b = threadIdx.x; b < B; b += blockDim.x) acc += partial[(long long)idx * B + b];
  for (int o = 16; o > 0; o >>= 1) acc += shfl_xor(acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    c128 t(0, 0);
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    out[idx] = t;
  }
}

// y[s] += sign * sum_i coef[s * ldc + i] * V_i[s]; the basis pointers and coefficients of
// the block's right-hand side are staged in shared memory, kAxpyMax at a time.  With out
// set (nv <= kAxpyMax), the result divided by nrm[s] goes to out[s] instead of y (zero
// when nrm[s] = 0): the projection and the normalisation of an Arnoldi step in one pass.
constexpr int kAxpyMax = 64;
template <typename T>
__global__ void axpy_multi(const c128* const* __restrict__ V, int nv, const c128* __restrict__ coef, int ldc,
                           double sign, c128* __restrict__ y, long long N, const double* __restrict__ nrm = nullptr,
                           c128* __restrict__ out = nullptr) {
  const int s = blockIdx.y;
  __shared__ const c128* sv[kAxpyMax];
  __shared__ Cx<T> sc[kAxpyMax];
  c128* ys = y + (long long)s * N;
  const T inv = (out && nrm[s] > 0) ? T(1.0 / nrm[s]) : T(0);
  for (int i0 = 0; i0 < nv; i0 += kAxpyMax) {
    const int nc = min(kAxpyMax, nv - i0);
    __syncthreads();
    for (int i = threadIdx.x; i < nc; i += blockDim.x) {
      sv[i] = V[i0 + i] + (long long)s * N;
      sc[i] = cvt<T>(sign * coef[(long long)s * ldc + i0 + i]);
    }
    __syncthreads();
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
      Cx<T> acc = cvt<T>(ys[p]);
      for (int i = 0; i < nc; ++i) cfma(acc, sc[i], cvt<T>(sv[i][p]));
      if (out) out[(long long)s * N + p] = cvt<double>(inv * acc);
      else ys[p] = cvt<double>(acc);
    }
  }
}

// v[s] = w[s] / nrm[s] (zero when nrm[s] = 0)
template <typename T>
__global__ void scale_kernel(const c128* __restrict__ w, const double* __restrict__ nrm, c128* __restrict__ v,
                             long long N) {
  const int s = blockIdx.y;
  const T a = nrm[s] > 0 ? T(1.0 / nrm[s]) : T(0);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x)
    v[s * N + p] = cvt<double>(a * cvt<T>(w[s * N + p]));
}

// dst[i] = src[i] for n 8-byte words (the mailbox transfers below)
__global__ void copy_words(const unsigned long long* __restrict__ src, unsigned long long* __restrict__ dst, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i];
}


}  // namespace

struct KrylovWork {
  int nrhs_cap = 0;
  std::vector<c128*> V;        // basis vectors, each [nrhs_cap][N]
  c128** d_V = nullptr;        // device copy of the pointer table
  int d_V_cap = 0;
  c128 *r = nullptr, *z = nullptr, *w = nullptr, *t = nullptr;
  c128* partial = nullptr;
  c128* dots = nullptr;        // [nrhs][vmax]
  c128* coef = nullptr;        // [nrhs][vmax]
  double* nrm = nullptr;       // [nrhs]
  int vmax = 0;
  // Mailbox for the solve's small host <-> device exchanges (Gram-Schmidt coefficients,
  // norms, pointer tables, the status word): mapped pinned host memory moved by a copy
  // kernel on the handle's stream instead of the copy engines, so that bulk transfers a
  // caller runs beside the solve on another stream (the next batch's right-hand sides, the
  // previous batch's solutions) never hold up its per-iteration exchanges.  Regions (bytes):
  // coefficients up, norms up, the basis table up, results down.
  unsigned char* mbox_h = nullptr;
  unsigned char* mbox_d = nullptr;
  size_t o_coef = 0, o_nrm = 0, o_vtab = 0, o_down = 0, mbox_bytes = 0;
};

// bytes (a multiple of 8) from host src to device dst through the mailbox region `region`;
// the region is rewritten only after a later stream synchronisation (the call sites below)
static int mbox_up(hsweep_s* h, size_t region, const void* src, void* dst, size_t bytes) {
  KrylovWork* k = h->kw;
  if (bytes == 0) return HSWEEP_OK;
  std::memcpy(k->mbox_h + region, src, bytes);
  const int nw = (int)(bytes / 8);
  copy_words<<<std::min(64, (nw + 255) / 256), 256, 0, h->stream>>>(
      reinterpret_cast<const unsigned long long*>(k->mbox_d + region), reinterpret_cast<unsigned long long*>(dst), nw);
  h->nlaunch += 1;
  HSW_CUDA(cudaGetLastError());
  return HSWEEP_OK;
}

// bytes (a multiple of 8) from device src to host dst; synchronises the stream
static int mbox_down(hsweep_s* h, const void* src, void* dst, size_t bytes) {
  KrylovWork* k = h->kw;
  if (bytes == 0) return HSWEEP_OK;
  const int nw = (int)(bytes / 8);
  copy_words<<<std::min(64, (nw + 255) / 256), 256, 0, h->stream>>>(
      reinterpret_cast<const unsigned long long*>(src), reinterpret_cast<unsigned long long*>(k->mbox_d + k->o_down), nw);
  h->nlaunch += 1;
  HSW_CUDA(cudaGetLastError());
  HSW_CUDA(cudaStreamSynchronize(h->stream));
  std::memcpy(dst, k->mbox_h + k->o_down, bytes);
  return HSWEEP_OK;
}

void hsw_krylov_free(hsweep_s* h) {
  if (!h->kw) return;
  KrylovWork* k = h->kw;
  for (c128* p : k->V) hsw_release(h, p);
  void* ptrs[] = {k->d_V, k->r, k->z, k->w, k->t, k->partial, k->dots, k->coef, k->nrm};
  for (void* p : ptrs) hsw_release(h, p);
  if (k->mbox_h) cudaFreeHost(k->mbox_h);
  delete k;
  h->kw = nullptr;
}

static int krylov_reserve(hsweep_s* h, int nrhs) {
  const int vmax = h->opt.gmres_max_it + 1;
  if (h->kw && h->kw->nrhs_cap >= nrhs) return HSWEEP_OK;
  hsw_krylov_free(h);
  KrylovWork* k = new (std::nothrow) KrylovWork();
  if (!k) return HSWEEP_ERR_OOM;
  h->kw = k;
  k->vmax = vmax;   // nrhs_cap is set last: a failed reservation leaves a workspace of capacity 0
  const size_t vb = (size_t)nrhs * h->N * sizeof(c128);
  int rc;
#define A(p, bytes) do { rc = hsw_alloc(h, (void**)&(p), (size_t)(bytes)); if (rc) return rc; } while (0)
  A(k->d_V, vmax * sizeof(c128*));
  A(k->r, vb); A(k->z, vb); A(k->w, vb); A(k->t, vb);
  A(k->partial, (size_t)nrhs * vmax * kRedBlocks * sizeof(c128));
  A(k->dots, (size_t)nrhs * vmax * sizeof(c128));
  A(k->coef, (size_t)nrhs * vmax * sizeof(c128));
  A(k->nrm, (size_t)nrhs * sizeof(double));
#undef A
  const size_t cb = ((size_t)nrhs * vmax * sizeof(c128) + 255) / 256 * 256;
  const size_t nb = ((size_t)nrhs * sizeof(double) + 255) / 256 * 256;
  const size_t vt = ((size_t)vmax * sizeof(c128*) + 255) / 256 * 256;
  k->o_coef = 0;
  k->o_nrm = cb;
  k->o_vtab = cb + nb;
  k->o_down = cb + nb + vt;
  k->mbox_bytes = k->o_down + cb;
  void* hp = nullptr;
  if (cudaHostAlloc(&hp, k->mbox_bytes, cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    return HSWEEP_ERR_OOM;
  }
  k->mbox_h = static_cast<unsigned char*>(hp);
  void* dp = nullptr;
  HSW_CUDA(cudaHostGetDevicePointer(&dp, hp, 0));
  k->mbox_d = static_cast<unsigned char*>(dp);
  k->nrhs_cap = nrhs;
  return HSWEEP_OK;
}

// basis vector i (allocated on first use)
static int basis(hsweep_s* h, int i, c128** out) {
  KrylovWork* k = h->kw;
  while ((int)k->V.size() <= i) {
    c128* p = nullptr;
    int rc = hsw_alloc(h, (void**)&p, (size_t)k->nrhs_cap * h->N * sizeof(c128));
    if (rc) return rc;
    k->V.push_back(p);
  }
  if (k->d_V_cap < (int)k->V.size()) {
    int rc = mbox_up(h, k->o_vtab, k->V.data(), k->d_V, k->V.size() * sizeof(c128*));
    if (rc) return rc;
    k->d_V_cap = (int)k->V.size();
  }
  *out = k->V[i];
  return HSWEEP_OK;
}

// <V_{first+i}[s], w[s]> for i < nv and, with with_norm, ||w[s]||^2 as entry nv, copied to
// host hd (nrhs x nt, nt = nv + with_norm); one read of w
static int batched_dots(hsweep_s* h, int first, int nv, const c128* w, int nrhs, std::vector<std::complex<double>>& hd,
                        bool lowp, bool with_norm = false) {
  KrylovWork* k = h->kw;
  const int nt = nv + (with_norm ? 1 : 0);
  if (lowp) dots_kernel<float><<<dim3(kRedBlocks, nrhs), 256, 0, h->stream>>>(k->d_V + first, nv, nt, w, h->N, k->partial);
  else dots_kernel<double><<<dim3(kRedBlocks, nrhs), 256, 0, h->stream>>>(k->d_V + first, nv, nt, w, h->N, k->partial);
  h->nlaunch += 1;
  reduce_partials<<<nrhs * nt, 256, 0, h->stream>>>(k->partial, kRedBlocks, k->dots);
  h->nlaunch += 1;
  HSW_CUDA(cudaGetLastError());
  hd.resize((size_t)nrhs * nt);
  return mbox_down(h, k->dots, hd.data(), (size_t)nrhs * nt * sizeof(c128));
}

// ||x[s]|| for every s, on the host
static int norms(hsweep_s* h, const c128* x, int nrhs, std::vector<double>& out, bool lowp = false) {
  KrylovWork* k = h->kw;
  if (lowp) sqnorm_kernel<float><<<dim3(kRedBlocks, nrhs), 256, 0, h->stream>>>(x, h->N, k->partial);
  else sqnorm_kernel<double><<<dim3(kRedBlocks, nrhs), 256, 0, h->stream>>>(x, h->N, k->partial);
  h->nlaunch += 1;
  reduce_partials<<<nrhs, 256, 0, h->stream>>>(k->partial, kRedBlocks, k->dots);
  h->nlaunch += 1;
  HSW_CUDA(cudaGetLastError());
  std::vector<std::complex<double>> hd(nrhs);
  int rc = mbox_down(h, k->dots, hd.data(), nrhs * sizeof(c128));
  if (rc) return rc;
  out.resize(nrhs);
  for (int s = 0; s < nrhs; ++s) out[s] = std::sqrt(std::max(0.0, hd[s].real()));
  return HSWEEP_OK;
}

static dim3 vec_grid(hsweep_s* h, int nrhs) {
  long long blocks = (h->N + 255) / 256;
  if (blocks > 1216) blocks = 1216;
  return dim3((unsigned)blocks, nrhs);
}

// Inner GMRES on (M A) d = z, x0 = 0, adding its solution d to u (the right-hand sides
// not active are left unchanged).  eta[s]: relative tolerance on ||z_s||; active[s]
// marks the right-hand sides being solved.  Adds the Arnoldi steps to iters.
static int gmres_inner(hsweep_s* h, const c128* z, int nrhs, const std::vector<double>& znrm,
                       const std::vector<double>& eta, std::vector<char>& active, c128* u, std::vector<int>& iters,
                       std::vector<double>& est) {
  KrylovWork* k = h->kw;
  const int maxit = h->opt.gmres_max_it;
  const long long N = h->N;
  // FP32 arithmetic on the FP64-stored vectors only when asked for (HSWEEP_MIXED)
  const bool lowp = h->prec == HSWEEP_MIXED && h->opt.krylov_lowp != 0;
  typedef std::complex<double> cd;
  std::vector<std::vector<cd>> H(nrhs, std::vector<cd>((size_t)(maxit + 1) * maxit, cd(0)));
  std::vector<std::vector<cd>> cs(nrhs, std::vector<cd>(maxit)), sn(nrhs, std::vector<cd>(maxit));
  std::vector<std::vector<cd>> g(nrhs, std::vector<cd>(maxit + 1, cd(0)));
  std::vector<int> ks(nrhs, 0);
  std::vector<char> run(active);
  for (int s = 0; s < nrhs; ++s) {
    g[s][0] = cd(znrm[s], 0);
    est[s] = 1.0;
    if (!(znrm[s] > 0)) run[s] = 0;
  }
  c128* v0;
  int rc = basis(h, 0, &v0);
  if (rc) return rc;
  {
    if ((rc = mbox_up(h, k->o_nrm, znrm.data(), k->nrm, nrhs * sizeof(double)))) return rc;
    if (lowp) scale_kernel<float><<<vec_grid(h, nrhs), 256, 0, h->stream>>>(z, k->nrm, v0, N);
    else scale_kernel<double><<<vec_grid(h, nrhs), 256, 0, h->stream>>>(z, k->nrm, v0, N);
    h->nlaunch += 1;
  }
  std::vector<cd> hd, hd2;
  int j = 0;
  for (; j < maxit; ++j) {
    bool any = false;
    for (int s = 0; s < nrhs; ++s) any |= run[s] != 0;
    if (!any) break;
    NvtxRange range("gmres step");
    c128 *vj, *vn;
    if ((rc = basis(h, j, &vj))) return rc;
    if ((rc = basis(h, j + 1, &vn))) return rc;
    // w = M (A v_j)
    if ((rc = hsw_matvec_prec(h, vj, k->t, nrhs, lowp))) return rc;
    if ((rc = hsw_apply(h, k->t, k->w, nrhs))) return rc;
    // classical Gram-Schmidt with selective re-orthogonalisation (Daniel, Gragg, Kaufman and
    // Stewart): the first pass reads w once for its projections and its norm; the norm after
    // the projection follows from Pythagoras, and a second pass runs (for the whole batch)
    // only when some right-hand side needs it: where more than half of the squared norm was
    // lost, except at the first step of an inner solve in FP64 arithmetic.  With several
    // basis vectors, classical Gram-Schmidt's loss of orthogonality compounds from step to
    // step (M A is close to the identity, so every step cancels most of w), and the usual
    // test is kept.  At the first step the basis is one vector and the loss is local: the new
    // vector keeps a component along it of about u sqrt(n0 / n1) (u the rounding of the dots,
    // n0 and n1 the squared norms before and after the projection), so a second pass runs
    // only where 1e-15 sqrt(n0 / n1) could exceed 1e-3 eta (n1 < (1e-12 / eta)^2 n0) or the
    // norm from Pythagoras, n0 - |h|^2, could lose more than 1e-8 of n1 (n1 < 1e-8 n0).
    std::vector<cd> hcol((size_t)nrhs * (j + 1), cd(0));
    std::vector<double> wn(nrhs, 0.0);
    bool second = false, fused = false;
    {
      if ((rc = batched_dots(h, 0, j + 1, k->w, nrhs, hd, lowp, true))) return rc;
      std::vector<cd> h1((size_t)nrhs * (j + 1));
      for (int s = 0; s < nrhs; ++s) {
        const double n0 = hd[(size_t)s * (j + 2) + j + 1].real();
        double n1 = n0;
        for (int i = 0; i <= j; ++i) {
          const cd v = hd[(size_t)s * (j + 2) + i];
          h1[(size_t)s * (j + 1) + i] = v;
          n1 -= std::norm(v);
        }
        if (run[s]) {
          const double q = eta[s] > 0 ? 1e-12 / eta[s] : 1.0;
          const double thr = (lowp || j > 0) ? 0.5 : std::min(0.5, std::max(q * q, 1e-8));
          if (!(n1 >= thr * n0)) second = true;
        }
        wn[s] = std::sqrt(std::max(0.0, n1));
      }
      for (size_t e = 0; e < h1.size(); ++e) hcol[e] += h1[e];
      if ((rc = mbox_up(h, k->o_coef, h1.data(), k->coef, h1.size() * sizeof(c128)))) return rc;
      // without a second pass the norm is known already: project and normalise in one pass
      fused = !second && j + 1 <= kAxpyMax;
      if (fused && (rc = mbox_up(h, k->o_nrm, wn.data(), k->nrm, nrhs * sizeof(double)))) return rc;
      const double* fn = fused ? k->nrm : nullptr;
      c128* fo = fused ? vn : nullptr;
      if (lowp)
        axpy_multi<float><<<vec_grid(h, nrhs), 256, 0, h->stream>>>(k->d_V, j + 1, k->coef, j + 1, -1.0, k->w, N, fn, fo);
      else
        axpy_multi<double><<<vec_grid(h, nrhs), 256, 0, h->stream>>>(k->d_V, j + 1, k->coef, j + 1, -1.0, k->w, N, fn, fo);
      h->nlaunch += 1;
    }
    if (second) {
      if ((rc = batched_dots(h, 0, j + 1, k->w, nrhs, hd, lowp))) return rc;
      for (size_t e = 0; e < hd.size(); ++e) hcol[e] += hd[e];
      if ((rc = mbox_up(h, k->o_coef, hd.data(), k->coef, hd.size() * sizeof(c128)))) return rc;
      if (lowp) axpy_multi<float><<<vec_grid(h, nrhs), 256, 0, h->stream>>>(k->d_V, j + 1, k->coef, j + 1, -1.0, k->w, N);
      else axpy_multi<double><<<vec_grid(h, nrhs), 256, 0, h->stream>>>(k->d_V, j + 1, k->coef, j + 1, -1.0, k->w, N);
      h->nlaunch += 1;
      if ((rc = norms(h, k->w, nrhs, wn, lowp))) return rc;
    }
    if (!fused) {
      if ((rc = mbox_up(h, k->o_nrm, wn.data(), k->nrm, nrhs * sizeof(double)))) return rc;
      if (lowp) scale_kernel<float><<<vec_grid(h, nrhs), 256, 0, h->stream>>>(k->w, k->nrm, vn, N);
      else scale_kernel<double><<<vec_grid(h, nrhs), 256, 0, h->stream>>>(k->w, k->nrm, vn, N);
      h->nlaunch += 1;
    }
    for (int s = 0; s < nrhs; ++s) {
      if (!run[s]) continue;
      cd* Hs = H[s].data();
      for (int i = 0; i <= j; ++i) Hs[i * maxit + j] = hcol[(size_t)s * (j + 1) + i];
      Hs[(j + 1) * maxit + j] = cd(wn[s], 0);
      for (int i = 0; i < j; ++i) {
        cd a = Hs[i * maxit + j], b = Hs[(i + 1) * maxit + j];
        Hs[i * maxit + j] = cs[s][i] * a + sn[s][i] * b;
        Hs[(i + 1) * maxit + j] = -std::conj(sn[s][i]) * a + std::conj(cs[s][i]) * b;
      }
      cd a = Hs[j * maxit + j], b = Hs[(j + 1) * maxit + j];
      double r = std::sqrt(std::norm(a) + std::norm(b));
      cs[s][j] = r != 0 ? std::conj(a) / r : cd(1);
      sn[s][j] = r != 0 ? std::conj(b) / r : cd(0);
      Hs[j * maxit + j] = cd(r, 0);
      Hs[(j + 1) * maxit + j] = 0;
      g[s][j + 1] = -std::conj(sn[s][j]) * g[s][j];
      g[s][j] = cs[s][j] * g[s][j];
      ks[s] = j + 1;
      iters[s] += 1;
      est[s] = std::abs(g[s][j + 1]) / znrm[s];
      if (est[s] <= eta[s] || wn[s] == 0.0 || r == 0.0) run[s] = 0;
    }
  }
  // u += sum_i y_i v_i with H y = g (upper-triangular back substitution per RHS; y = 0
  // for the right-hand sides not active)
  std::vector<cd> Y((size_t)nrhs * std::max(1, maxit), cd(0));
  int kmax = 0;
  for (int s = 0; s < nrhs; ++s) {
    if (!active[s]) continue;
    const int kk = ks[s];
    kmax = std::max(kmax, kk);
    cd* Hs = H[s].data();
    for (int i = kk - 1; i >= 0; --i) {
      cd acc = g[s][i];
      for (int l = i + 1; l < kk; ++l) acc -= Hs[i * maxit + l] * Y[(size_t)s * maxit + l];
      Y[(size_t)s * maxit + i] = Hs[i * maxit + i] != cd(0) ? acc / Hs[i * maxit + i] : cd(0);
    }
  }
  if (kmax > 0) {
    std::vector<cd> Yc((size_t)nrhs * kmax, cd(0));
    for (int s = 0; s < nrhs; ++s)
      for (int i = 0; i < kmax; ++i) Yc[(size_t)s * kmax + i] = Y[(size_t)s * maxit + i];
    if ((rc = mbox_up(h, k->o_coef, Yc.data(), k->coef, Yc.size() * sizeof(c128)))) return rc;
    // u is FP64 in every mode: the update runs in FP64
    axpy_multi<double><<<vec_grid(h, nrhs), 256, 0, h->stream>>>(k->d_V, kmax, k->coef, kmax, 1.0, u, N);
    h->nlaunch += 1;
    HSW_CUDA(cudaGetLastError());
  }
  HSW_CUDA(cudaStreamSynchronize(h->stream));
  return HSWEEP_OK;
}

int hsw_solve(hsweep_s* h, const c128* f, c128* u, int nrhs, double tol, int* iters_out, double* relres_out) {
  int rc = krylov_reserve(h, nrhs);
  if (rc) return rc;
  KrylovWork* k = h->kw;
  const long long N = h->N;
  const bool mixed = h->prec == HSWEEP_MIXED;
  const bool lowp = mixed && h->opt.krylov_lowp != 0;
  std::vector<int> iters(nrhs, 0);
  std::vector<double> Mfn, fn, zn, est(nrhs, 1.0);
  // ||M f|| (the reference of the stopping test) and ||f||
  if ((rc = hsw_apply(h, f, k->z, nrhs))) return rc;
  if ((rc = norms(h, k->z, nrhs, Mfn, lowp))) return rc;
  if ((rc = norms(h, f, nrhs, fn))) return rc;
  // with a zero initial guess the first residual is f itself and M r = M f is at hand
  std::vector<double> un;
  if ((rc = norms(h, u, nrhs, un))) return rc;
  bool u_zero = true;
  for (int s = 0; s < nrhs; ++s) u_zero = u_zero && un[s] == 0.0;
  std::vector<char> done(nrhs, 0);
  const int outer_max = h->opt.refine_max;
  bool all_done = false;
  for (int outer = 0; outer < outer_max && !all_done; ++outer) {
    // r = f - A u, z = M r
    if (outer == 0 && u_zero) {
      zn = Mfn;      // k->z still holds M f
    } else {
      if ((rc = hsw_residual(h, f, u, k->r, nrhs))) return rc;
      if ((rc = hsw_apply(h, k->r, k->z, nrhs))) return rc;
      if ((rc = norms(h, k->z, nrhs, zn, lowp))) return rc;
    }
    std::vector<char> active(nrhs, 0);
    std::vector<double> eta(nrhs, 0.0);
    all_done = true;
    for (int s = 0; s < nrhs; ++s) {
      if (!(zn[s] > tol * Mfn[s])) { done[s] = 1; continue; }
      done[s] = 0;
      active[s] = 1;
      all_done = false;
      const double need = tol * Mfn[s] / zn[s];
      // in HSWEEP_MIXED the complex64 sweeps leave M A accurate to a few 1e-7, so the inner
      // solve is asked for no more than a relative 4e-6 and the refinement does the rest
      eta[s] = mixed ? std::max(0.5 * need, 4e-6) : 0.9 * need;
    }
    if (all_done) break;
    // u += d for the active right-hand sides
    if ((rc = gmres_inner(h, k->z, nrhs, zn, eta, active, u, iters, est))) return rc;
    if (!mixed) {
      // FP64: the inner residual estimate is the FP64 one; stop when it met the tolerance
      bool ok = true;
      for (int s = 0; s < nrhs; ++s)
        if (active[s] && !(est[s] * zn[s] <= tol * Mfn[s])) ok = false;
      if (ok) { all_done = true; for (int s = 0; s < nrhs; ++s) done[s] = 1; }
    } else {
      // HSWEEP_MIXED: the inner estimate is exact up to the complex64 sweep's departure from
      // a linear map, at most kSweepNoise times ||z||; once ||z|| is small enough that this
      // departure is below half the tolerance, an inner solve that met half the tolerance
      // ends the refinement without another apply to re-measure ||M r||
      bool ok = true;
      for (int s = 0; s < nrhs; ++s)
        if (active[s] && !(zn[s] * kSweepNoise <= 0.5 * tol * Mfn[s] && est[s] * zn[s] <= 0.5 * tol * Mfn[s]))
          ok = false;
      if (ok) { all_done = true; for (int s = 0; s < nrhs; ++s) done[s] = 1; }
    }
  }
  // final FP64 residual
  if ((rc = hsw_residual(h, f, u, k->r, nrhs))) return rc;
  std::vector<double> rn;
  if ((rc = norms(h, k->r, nrhs, rn))) return rc;
  if (!all_done && mixed) {
    if ((rc = hsw_apply(h, k->r, k->z, nrhs))) return rc;
    if ((rc = norms(h, k->z, nrhs, zn, lowp))) return rc;
    all_done = true;
    for (int s = 0; s < nrhs; ++s) if (!(zn[s] <= tol * Mfn[s])) all_done = false;
  }
  for (int s = 0; s < nrhs; ++s) {
    if (iters_out) iters_out[s] = iters[s];
    if (relres_out) relres_out[s] = fn[s] > 0 ? rn[s] / fn[s] : 0.0;
  }
  int st[2] = {0, -1};
  if ((rc = mbox_down(h, h->d_status, st, sizeof(st)))) return rc;
  if (st[0] != 0) return st[0];
  return all_done ? HSWEEP_OK : HSWEEP_ERR_NOT_CONVERGED;
}
