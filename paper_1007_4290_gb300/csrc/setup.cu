// The setup sweep of Algorithm 2.5 on the GPU: for m = 1..n
//   S~_m = A_mm - A_{m,m-1} T~_{m-1} A_{m-1,m}   (hdiagmul + hsub; Section 2.3)
//   T~_m = hinv(S~_m)
// with every matrix a weakly admissible H-matrix in symmetric storage (siblings a, b:
// block (a, b) = F_a F_b^t, block (b, a) = F_b F_a^t; dense leaves).
//
// hinv is organised level by level, bottom-up, instead of the paper's depth-first
// 2 x 2 recursion; both give the same inverse before truncation.  For a node t with
// children a, b and S(a, b) = U V^t:
//     S_t = diag(S_a, S_b) + P C P^t,  P = diag(U, V),  C = [[0, I], [I, 0]],
// so by the Woodbury identity, with G_a = S_a^{-1} and G_b = S_b^{-1} already built,
//     Y = diag(G_a U, G_b V),  M = [[U^t Y_a, I], [I, V^t Y_b]]^{-1},
//     S_t^{-1} = diag(G_a, G_b) - Y M Y^t.
// The new off-diagonal block is -Y_a M12 Y_b^t; the diagonal corrections -Y_a M11 Y_a^t
// and -Y_b M22 Y_b^t are rank-k updates of every block below a and b ("hadd" with a
// factorised term).  All nodes of one depth are processed by the same launches.
// Recompression ("Matrix addition": QR of both factors, SVD of the small core,
// truncation at eps_H relative to the block's largest singular value, at most r_max
// terms) runs once per layer, after the last depth, on every block whose final core fits
// the SVD's shared memory: appended columns accumulate (up to depth x (r_max + 1) of
// them), the untruncated factors feed the products of the higher depths, and each block
// is truncated once, in its final form.  Blocks whose core would not fit (large blocks
// in complex128) are recompressed after every depth that changed them.  A small block whose factors have at least as
// many columns as rows takes the dense path: its core is the block itself, C = F_a F_b^t,
// and its new factors come straight from the SVD of C (no QR).  QR is classical
// Gram-Schmidt with re-orthogonalisation; the SVD is one-sided (Hestenes) Jacobi.
// The leaf inverses are computed in FP64 with partial pivoting in both precisions.
#include <algorithm>
#include <cmath>
#include <utility>
#include "handle.h"

namespace {

constexpr int kBlk = 256;

template <typename R> struct Tiny;
template <> struct Tiny<double> {
  static constexpr double dep = 1e-13;    // Gram-Schmidt: dependent-column threshold
  static constexpr double jac = 1e-15;    // Jacobi: orthogonality tolerance (about 8 ulp)
  static constexpr double neg = 1e-28;    // Jacobi: squared norm of a rounding-noise column
                                          // (normalised: below 1e-14 of the largest column)
};
template <> struct Tiny<float> {
  static constexpr float dep = 2e-6f;
  static constexpr float jac = 4e-7f;     // about 7 ulp: tighter only rotates rounding noise
  static constexpr float neg = 1e-14f;    // below 1e-7 of the largest column: FP32 noise
};

template <typename R> __device__ __forceinline__ Cx<R> warp_sum(Cx<R> v) {
  for (int o = 16; o > 0; o >>= 1) v += shfl_xor(v, o);
  return v;
}
template <typename R> __device__ __forceinline__ R warp_sum_r(R v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of a real value (result broadcast to all threads).
template <typename R> __device__ R block_sum(R v, R* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum_r(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  R t = 0;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

struct Geo {          // tree and buffer geometry passed by value to every kernel
  int n, L, leaf, nnodes, r_max, KCAP, WCAP, QCAP;
  const int* lo;
  const int* sz;
  const int* rowleaf;      // [n] leaf node of each row
  const long long* sfo;    // S factor offsets (capacity KCAP per node)
  const long long* gfo;    // G factor offsets (capacity cap[v] columns per node)
  const int* cap;          // column capacity of every node's G factor
  const long long* qro;    // offsets of the reductions Qr (cap[v] x KCAP per node)
  const long long* rbo;    // offsets of the R factors (min(sz, cap) x cap, row-major, ld cap)
  const int* list;         // recompression kernels: the nodes (or left siblings) to process
};

__device__ __forceinline__ int depth_of(int v) { return 31 - __clz(v); }

// ---------------------------------------------------------------------------------
// S~_m: leaves A_mm[leaf] - D T_leaf D, factors [-D F_a, a e_last] / [D F_b, e_first].
template <typename R>
__global__ void schur_leaves(Geo g, int m, const c128* __restrict__ diag, const c128* __restrict__ east,
                             const c128* __restrict__ north, const Cx<R>* __restrict__ Tprev,
                             Cx<R>* __restrict__ S_leaf) {
  const int lam = (1 << g.L) + blockIdx.x;
  const int lo = g.lo[lam], s = g.sz[lam], lf = g.leaf;
  for (int e = threadIdx.x; e < lf * lf; e += blockDim.x) {
    const int a = e % lf, b = e / lf;     // column-major: entry (a, b) at b*leaf + a
    Cx<R> v(0, 0);
    if (a < s && b < s) {
      const int i = lo + a, j = lo + b;
      c128 av(0, 0);
      if (a == b) av = diag[(long long)m * g.n + i];
      else if (j == i + 1) av = east[(long long)m * (g.n + 1) + j];
      else if (i == j + 1) av = east[(long long)m * (g.n + 1) + i];
      v = cvt<R>(av);
      if (Tprev) {
        Cx<R> di = cvt<R>(north[(long long)m * g.n + i]), dj = cvt<R>(north[(long long)m * g.n + j]);
        v -= di * (Tprev[(long long)blockIdx.x * lf * lf + e] * dj);
      }
    } else if (a == b) {
      v = Cx<R>(1, 0);    // identity padding keeps the padded leaf invertible
    }
    S_leaf[(long long)blockIdx.x * lf * lf + e] = v;
  }
}

template <typename R>
__global__ void schur_factors(Geo g, int m, const c128* __restrict__ east, const c128* __restrict__ north,
                              const Cx<R>* __restrict__ Tprev, const long long* __restrict__ toff,
                              const int* __restrict__ trank, Cx<R>* __restrict__ S_F, int* __restrict__ S_rank) {
  const int v = 2 + blockIdx.x;
  const int lo = g.lo[v], s = g.sz[v];
  const bool left = (v & 1) == 0;
  const int r0 = Tprev ? trank[v] : 0;
  const int k = r0 + 1;
  Cx<R>* dst = S_F + g.sfo[v];
  const int edge = g.lo[v | 1];     // the coupling edge joins rows edge-1 and edge
  for (int e = threadIdx.x; e < s * k; e += blockDim.x) {
    const int i = e % s, col = e / s;
    Cx<R> val(0, 0);
    if (col < r0) {
      Cx<R> dv = cvt<R>(north[(long long)m * g.n + lo + i]);
      val = dv * Tprev[toff[v] + (long long)col * s + i];
      if (left) val = -val;
    } else {
      // the rank-one coupling a e_last e_first^t, split as sqrt(a) on both sides so
      // that the two factors carry the same scale
      const c128 ra = csqrt(east[(long long)m * (g.n + 1) + edge]);
      if (left) { if (i == s - 1) val = cvt<R>(ra); }
      else if (i == 0) val = cvt<R>(ra);
    }
    dst[(long long)col * s + i] = val;
  }
  if (threadIdx.x == 0) S_rank[v] = k;
}

// ---------------------------------------------------------------------------------
// Leaf inverses, FP64 Gauss-Jordan with partial pivoting (one block per leaf).
template <typename R>
__global__ void leaf_inverse(Geo g, int m, const Cx<R>* __restrict__ S_leaf, Cx<R>* __restrict__ G_leaf,
                             int* status) {
  __shared__ c128 A[8][16];
  __shared__ c128 colk[8];
  __shared__ int piv;
  const int lf = g.leaf;
  const Cx<R>* src = S_leaf + (long long)blockIdx.x * lf * lf;
  for (int e = threadIdx.x; e < lf * 2 * lf; e += blockDim.x) {
    int a = e / (2 * lf), b = e % (2 * lf);
    A[a][b] = b < lf ? cvt<double>(src[b * lf + a]) : c128(a == b - lf ? 1.0 : 0.0, 0.0);
  }
  __shared__ double s_red[4];
  __syncthreads();
  // the largest squared modulus of the leaf's entries (one entry per thread, then warps)
  double scale2 = 0;
  for (int e = threadIdx.x; e < lf * lf; e += blockDim.x) scale2 = fmax(scale2, abs2(A[e / lf][e % lf]));
  for (int o = 16; o > 0; o >>= 1) scale2 = fmax(scale2, __shfl_xor_sync(0xffffffffu, scale2, o));
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = scale2;
  __syncthreads();
  scale2 = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) scale2 = fmax(scale2, s_red[i]);
  bool bad = false;
  for (int k = 0; k < lf; ++k) {
    if (threadIdx.x == 0) {
      int p = k;
      double best = abs2(A[k][k]);
      for (int a = k + 1; a < lf; ++a)
        if (abs2(A[a][k]) > best) { best = abs2(A[a][k]); p = a; }
      piv = p;
    }
    __syncthreads();
    const int p = piv;
    if (p != k && threadIdx.x < 2 * lf) {
      c128 t = A[k][threadIdx.x]; A[k][threadIdx.x] = A[p][threadIdx.x]; A[p][threadIdx.x] = t;
    }
    __syncthreads();
    const c128 pv = A[k][k];
    if (!(abs2(pv) > 1e-28 * scale2)) { bad = true; break; }   // |pivot| <= 1e-14 max |entry|
    const c128 ip = cinv(pv);
    __syncthreads();
    if (threadIdx.x < 2 * lf) A[k][threadIdx.x] = A[k][threadIdx.x] * ip;
    if (threadIdx.x < lf) colk[threadIdx.x] = A[threadIdx.x][k];
    __syncthreads();
    for (int e = threadIdx.x; e < lf * 2 * lf; e += blockDim.x) {
      int a = e / (2 * lf), b = e % (2 * lf);
      if (a != k) A[a][b] = A[a][b] - colk[a] * A[k][b];
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) report_error(status, HSWEEP_ERR_NUMERIC, m);
    return;
  }
  Cx<R>* dst = G_leaf + (long long)blockIdx.x * lf * lf;
  for (int e = threadIdx.x; e < lf * lf; e += blockDim.x) {
    int a = e % lf, b = e / lf;
    dst[e] = cvt<R>(A[a][lf + b]);
  }
}

// ---------------------------------------------------------------------------------
// Y_v = G_v X_v for every node v at depth d+1 (X_v = S factor of v, k_v columns):
// an H-matrix times a tall-skinny block, as reductions (per node u below depth d+1:
// Qr_u = F_u^t X restricted to u) followed by an expansion.
template <typename R>
__global__ void tsmm_reduce(Geo g, int d, const Cx<R>* __restrict__ G_F, const int* __restrict__ G_rank,
                            const Cx<R>* __restrict__ S_F, const int* __restrict__ S_rank, Cx<R>* __restrict__ Qr) {
  const int u = (1 << (d + 2)) + blockIdx.x;
  const int du = depth_of(u);
  const int nu = u >> (du - (d + 1));          // ancestor at depth d+1
  const int ru = G_rank[u], k = S_rank[nu];
  const int s = g.sz[u], ld_x = g.sz[nu], xo = g.lo[u] - g.lo[nu];
  const Cx<R>* F = G_F + g.gfo[u];
  const Cx<R>* X = S_F + g.sfo[nu];
  Cx<R>* out = Qr + g.qro[u];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int kr = warp; kr < ru; kr += nw) {
    for (int c0 = 0; c0 < k; c0 += 8) {
      Cx<R> acc[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) acc[t] = Cx<R>(0, 0);
      for (int i = lane; i < s; i += 32) {
        Cx<R> f = F[(long long)kr * s + i];
#pragma unroll
        for (int t = 0; t < 8; ++t)
          if (c0 + t < k) cfma(acc[t], f, X[(long long)(c0 + t) * ld_x + xo + i]);
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        Cx<R> v = warp_sum(acc[t]);
        if (lane == 0 && c0 + t < k) out[kr * g.KCAP + c0 + t] = v;
      }
    }
  }
}

template <typename R>
__global__ void tsmm_expand(Geo g, int d, const Cx<R>* __restrict__ G_leaf, const Cx<R>* __restrict__ G_F,
                            const int* __restrict__ G_rank, const Cx<R>* __restrict__ S_F,
                            const int* __restrict__ S_rank, const Cx<R>* __restrict__ Qr, Cx<R>* __restrict__ Y) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int col = blockIdx.y;
  if (row >= g.n) return;
  const int lam = g.rowleaf[row];
  const int nu = lam >> (g.L - (d + 1));
  const int k = S_rank[nu];
  if (col >= k) return;
  const int lo_nu = g.lo[nu], ld = g.sz[nu];
  const Cx<R>* X = S_F + g.sfo[nu] + (long long)col * ld;
  Cx<R> y(0, 0);
  {
    const int lf = g.leaf, a = row - g.lo[lam], s = g.sz[lam];
    const Cx<R>* D = G_leaf + (long long)(lam - (1 << g.L)) * lf * lf;
    for (int b = 0; b < s; ++b) cfma(y, D[b * lf + a], X[g.lo[lam] - lo_nu + b]);
  }
  for (int du = d + 2; du <= g.L; ++du) {
    const int u = lam >> (g.L - du);
    const int ru = G_rank[u];
    const Cx<R>* F = G_F + g.gfo[u] + (row - g.lo[u]);
    const Cx<R>* q = Qr + g.qro[u ^ 1] + col;
    const int s = g.sz[u];
    for (int kr = 0; kr < ru; ++kr) cfma(y, F[(long long)kr * s], q[kr * g.KCAP]);
  }
  Y[(long long)lo_nu * g.KCAP + (long long)col * ld + (row - lo_nu)] = y;
}

// ---------------------------------------------------------------------------------
// Woodbury core per node t at depth d: P = U^t Y_a, Q = V^t Y_b (k x k), then
// M = [[P, I], [I, Q]]^{-1} by in-place Gauss-Jordan with partial pivoting.
template <typename R>
__global__ void core_dots(Geo g, int d, const Cx<R>* __restrict__ S_F, const int* __restrict__ S_rank,
                          const Cx<R>* __restrict__ Y, Cx<R>* __restrict__ PQ) {
  const int t = (1 << d) + blockIdx.x / 2;
  const int side = blockIdx.x & 1;
  const int v = 2 * t + side;
  const int k = S_rank[v], s = g.sz[v];
  const Cx<R>* U = S_F + g.sfo[v];
  const Cx<R>* Yv = Y + (long long)g.lo[v] * g.KCAP;
  Cx<R>* out = PQ + ((long long)(t - (1 << d)) * 2 + side) * g.KCAP * g.KCAP;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int e = blockIdx.y * nw + warp; e < k * k; e += gridDim.y * nw) {
    const int a = e / k, b = e % k;
    Cx<R> acc(0, 0);
    for (int i = lane; i < s; i += 32) cfma(acc, U[(long long)a * s + i], Yv[(long long)b * s + i]);
    acc = warp_sum(acc);
    if (lane == 0) out[a * g.KCAP + b] = acc;
  }
}

template <typename R>
__global__ void core_inverse(Geo g, int d, int m, const int* __restrict__ S_rank, const Cx<R>* __restrict__ PQ,
                             Cx<R>* __restrict__ Mb, int* status) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int t = (1 << d) + blockIdx.x;
  const int k = S_rank[2 * t];
  const int n2 = 2 * k;
  Cx<R>* A = reinterpret_cast<Cx<R>*>(sm);                 // n2 x n2, row-major
  R* red = reinterpret_cast<R*>(A + n2 * n2);              // [32]
  int* piv = reinterpret_cast<int*>(red + 32);             // [n2]
  __shared__ int s_p;
  __shared__ R s_best;
  const Cx<R>* P = PQ + ((long long)(t - (1 << d)) * 2) * g.KCAP * g.KCAP;
  const Cx<R>* Q = P + g.KCAP * g.KCAP;
  for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {
    const int a = e / n2, b = e % n2;
    Cx<R> v(0, 0);
    if (a < k && b < k) v = P[a * g.KCAP + b];
    else if (a >= k && b >= k) v = Q[(a - k) * g.KCAP + (b - k)];
    else if (a < k && b == a + k) v = Cx<R>(1, 0);
    else if (a >= k && b == a - k) v = Cx<R>(1, 0);
    A[e] = v;
  }
  R mx = 0;
  for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) mx = fmax(mx, abs2(A[e]));
  __syncthreads();
  // block max
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    mx = 0;
    for (int i = 0; i < nw; ++i) mx = fmax(mx, red[i]);
    __syncthreads();
  }
  const R tiny = (sizeof(R) == 8 ? R(1e-30) : R(1e-14)) * mx;   // on |pivot|^2
  bool bad = false;
  // Gauss-Jordan in place, three block barriers per column: (1) pivot search and the
  // pivot's inverse, (2) the row interchange with the normalisation of the pivot row, (3)
  // the elimination of the other rows, each row owned by a group of gT lanes of one warp
  // (the group reads its multiplier, synchronises, then updates its columns, the pivot
  // column included)
  int gT = 1;
  while (gT < 32 && 2 * gT * n2 <= (int)blockDim.x) gT *= 2;
  const int rows_per_pass = (int)blockDim.x / gT;
  __shared__ Cx<R> s_ip;
  for (int kk = 0; kk < n2; ++kk) {
    if (threadIdx.x < 32) {
      // partial pivoting: warp 0 finds the largest |A[a][kk]|, a >= kk (ties: the smallest a)
      int p = n2;
      R best = R(-1);
      for (int a = kk + (int)threadIdx.x; a < n2; a += 32) {
        const R v = abs2(A[a * n2 + kk]);
        if (v > best) { best = v; p = a; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const R ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, p, o);
        if (ob > best || (ob == best && op < p)) { best = ob; p = op; }
      }
      if (threadIdx.x == 0) {
        s_p = p;
        s_best = best;
        piv[kk] = p;
        if (best > tiny) s_ip = cinv(A[p * n2 + kk]);
      }
    }
    __syncthreads();                                                     // (1)
    if (!(s_best > tiny)) { bad = true; break; }
    const int p = s_p;
    const Cx<R> ip = s_ip;
    for (int b = threadIdx.x; b < n2; b += blockDim.x) {
      const Cx<R> tk = A[kk * n2 + b], tp = A[p * n2 + b];
      if (p != kk) A[p * n2 + b] = tk;
      A[kk * n2 + b] = ((b == kk) ? Cx<R>(1, 0) : tp) * ip;
    }
    __syncthreads();                                                     // (2)
    for (int a0 = 0; a0 < n2; a0 += rows_per_pass) {
      const int a = a0 + (int)threadIdx.x / gT, sub = (int)threadIdx.x % gT;
      const bool live = a < n2 && a != kk;
      const Cx<R> f = live ? A[a * n2 + kk] : Cx<R>(0, 0);
      __syncwarp();
      if (live)
        for (int b = sub; b < n2; b += gT)
          A[a * n2 + b] = (b == kk) ? -(f * ip) : A[a * n2 + b] - f * A[kk * n2 + b];
    }
    __syncthreads();                                                     // (3)
  }
  if (bad) {
    if (threadIdx.x == 0) report_error(status, HSWEEP_ERR_NUMERIC, m);
    return;
  }
  // undo the row interchanges as column interchanges, in reverse order
  for (int kk = n2 - 1; kk >= 0; --kk) {
    const int p = piv[kk];
    if (p != kk)
      for (int a = threadIdx.x; a < n2; a += blockDim.x) {
        Cx<R> tmp = A[a * n2 + kk]; A[a * n2 + kk] = A[a * n2 + p]; A[a * n2 + p] = tmp;
      }
    __syncthreads();
  }
  Cx<R>* M = Mb + (long long)(t - (1 << d)) * 4 * g.KCAP * g.KCAP;
  for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {
    const int a = e / n2, b = e % n2;
    M[a * 2 * g.KCAP + b] = A[e];
  }
}

// W_v = Y_v M_side (k x k block of M), and the new off-diagonal block at the parent:
// F_a = -Y_a M12, F_b = Y_b.
template <typename R>
__global__ void woodbury_form(Geo g, int d, const int* __restrict__ S_rank, const Cx<R>* __restrict__ Y,
                              const Cx<R>* __restrict__ Mb, Cx<R>* __restrict__ W, Cx<R>* __restrict__ G_F,
                              int* __restrict__ G_rank) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int col = blockIdx.y;
  if (row >= g.n) return;
  const int v = g.rowleaf[row] >> (g.L - (d + 1));
  const int t = v >> 1, side = v & 1;
  const int k = S_rank[v];
  if (col >= k) return;
  const int s = g.sz[v], i = row - g.lo[v];
  const Cx<R>* Yv = Y + (long long)g.lo[v] * g.KCAP;
  const Cx<R>* M = Mb + (long long)(t - (1 << d)) * 4 * g.KCAP * g.KCAP;
  const int ldm = 2 * g.KCAP;
  const int off = side ? k : 0;
  Cx<R> w(0, 0), nf(0, 0);
  for (int j = 0; j < k; ++j) {
    const Cx<R> y = Yv[(long long)j * s + i];
    cfma(w, y, M[(off + j) * ldm + off + col]);          // M11 or M22
    if (!side) cfma(nf, y, M[j * ldm + k + col]);         // M12
  }
  W[(long long)g.lo[v] * g.KCAP + (long long)col * s + i] = w;
  Cx<R>* F = G_F + g.gfo[v];
  F[(long long)col * s + i] = side ? Yv[(long long)col * s + i] : -nf;
  if (i == 0 && col == 0) G_rank[v] = k;
}

// Append the rank-k correction to every node below depth d+1 and update the leaves
// (a leaf at depth d+1 itself only gets the dense update; its factor slot holds the
// new block written by woodbury_form).
template <typename R>
__global__ void woodbury_append(Geo g, int d, const int* __restrict__ S_rank, const Cx<R>* __restrict__ Y,
                                const Cx<R>* __restrict__ W, Cx<R>* __restrict__ G_F, int* __restrict__ G_rank,
                                Cx<R>* __restrict__ G_leaf) {
  const int u = (1 << (d + 1)) + blockIdx.x;
  const int du = depth_of(u);
  const int nu = u >> (du - (d + 1));
  const int k = S_rank[nu];
  const bool append = du >= d + 2;
  const int r0 = append ? G_rank[u] : 0;
  const int s = g.sz[u], ld = g.sz[nu], xo = g.lo[u] - g.lo[nu];
  const Cx<R>* Yv = Y + (long long)g.lo[nu] * g.KCAP;
  const Cx<R>* Wv = W + (long long)g.lo[nu] * g.KCAP;
  const bool left = (u & 1) == 0;
  Cx<R>* F = G_F + g.gfo[u];
  if (append)
    for (int e = threadIdx.x; e < s * k; e += blockDim.x) {
      const int i = e % s, j = e / s;
      F[(long long)(r0 + j) * s + i] = left ? -Wv[(long long)j * ld + xo + i] : Yv[(long long)j * ld + xo + i];
    }
  if (du == g.L) {     // leaf: G_leaf -= W[leaf] Y[leaf]^t
    const int lf = g.leaf;
    Cx<R>* D = G_leaf + (long long)(u - (1 << g.L)) * lf * lf;
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
      const int a = e % s, b = e / s;
      Cx<R> acc(0, 0);
      for (int j = 0; j < k; ++j) cfma(acc, Wv[(long long)j * ld + xo + a], Yv[(long long)j * ld + xo + b]);
      D[b * lf + a] -= acc;
    }
  }
  __syncthreads();
  if (append && threadIdx.x == 0) G_rank[u] = r0 + k;
}

// ---------------------------------------------------------------------------------
// Recompression, step 1, for the nodes u = list[blockIdx.x]: with w = rank(u) columns,
// a factor with at least as many columns as rows (w >= sz(u)) takes the dense path,
// Q = I and R = F_u (qcols = sz(u), qmode = 1); otherwise Gram-Schmidt QR (twice
// orthogonalised) of F_u in place, the Q columns compacted to the independent ones and
// R (qc x w) written out (qmode = 0).  R is row-major with leading dimension cap(u).  When
// F_u fits the kernel's shared memory (qs_entries), the orthogonalisation runs there and
// the kept columns are written back at the end (every projection reads all earlier
// columns: O(w^2 s) reads that would otherwise go to L2).
template <typename R>
__global__ void qr_cgs2(Geo g, Cx<R>* __restrict__ G_F, const int* __restrict__ G_rank, Cx<R>* __restrict__ Rb,
                        int* __restrict__ qcols, int* __restrict__ qmode, int qs_entries) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int u = g.list[blockIdx.x];
  const int s = g.sz[u], w = G_rank[u], ld = g.cap[u];
  Cx<R>* F = G_F + g.gfo[u];
  Cx<R>* Rm = Rb + g.rbo[u];                               // row-major qc x w, ld cap(u)
  if (w >= s && s <= g.QCAP) {
    for (int e = threadIdx.x; e < s * w; e += blockDim.x) {
      const int i = e % s, l = e / s;
      Rm[(long long)i * ld + l] = F[e];
    }
    if (threadIdx.x == 0) { qcols[u] = s; qmode[u] = 1; }
    return;
  }
  Cx<R>* v = reinterpret_cast<Cx<R>*>(sm);                // [s]
  Cx<R>* c = v + s;                                        // [QCAP]
  R* red = reinterpret_cast<R*>(c + g.QCAP);               // [32]
  const size_t qs_off = ((size_t)(s + g.QCAP) * sizeof(Cx<R>) + 32 * sizeof(R) + 15) & ~size_t(15);
  const bool qsh = (long long)s * w <= qs_entries;
  Cx<R>* Fq = qsh ? reinterpret_cast<Cx<R>*>(sm + qs_off) : F;   // the columns being orthogonalised
  __shared__ int s_qc;
  if (threadIdx.x == 0) s_qc = 0;
  const int rows = min(s, ld);
  for (int e = threadIdx.x; e < rows * w; e += blockDim.x) Rm[(long long)(e / w) * ld + e % w] = Cx<R>(0, 0);
  if (qsh)
    for (int e = threadIdx.x; e < s * w; e += blockDim.x) Fq[e] = F[e];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  // lanes per row of the projection update: a power of two, at most 32 and at most
  // blockDim / s (at least 1); blockDim.x is a multiple of 32
  int gT = 1;
  while (gT < 32 && 2 * gT * s <= (int)blockDim.x) gT *= 2;
  const int rows_per_pass = (int)blockDim.x / gT;
  for (int j = 0; j < w; ++j) {
    const int qc = s_qc;
    R nrm0 = 0;
    for (int i = threadIdx.x; i < s; i += blockDim.x) {
      v[i] = Fq[(long long)j * s + i];
      nrm0 += abs2(v[i]);
    }
    nrm0 = block_sum(nrm0, red);
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int l = warp; l < qc; l += nw) {
        Cx<R> acc(0, 0);
        for (int i = lane; i < s; i += 32) cfma_conj(acc, Fq[(long long)l * s + i], v[i]);
        acc = warp_sum(acc);
        if (lane == 0) {
          c[l] = acc;
          Rm[(long long)l * ld + j] += acc;
        }
      }
      __syncthreads();
      // v -= Q c: gT lanes per row share the sum over the kept columns (all threads busy
      // when the block has fewer rows than threads)
      for (int i0 = 0; i0 < s; i0 += rows_per_pass) {
        const int i = i0 + threadIdx.x / gT, sub = threadIdx.x % gT;
        Cx<R> acc(0, 0);
        if (i < s)
          for (int l = sub; l < qc; l += gT) cfma(acc, Fq[(long long)l * s + i], c[l]);
        for (int o = gT >> 1; o > 0; o >>= 1) acc += shfl_xor(acc, o);
        if (i < s && sub == 0) v[i] -= acc;
      }
      __syncthreads();
    }
    R nr = 0;
    for (int i = threadIdx.x; i < s; i += blockDim.x) nr += abs2(v[i]);
    nr = block_sum(nr, red);
    if (nr > Tiny<R>::dep * Tiny<R>::dep * nrm0 && nr > 0) {
      const R sn = sqrt(nr), is = R(1) / sn;
      for (int i = threadIdx.x; i < s; i += blockDim.x) Fq[(long long)qc * s + i] = is * v[i];
      if (threadIdx.x == 0) {
        Rm[(long long)qc * ld + j] = Cx<R>(sn, 0);
        s_qc = qc + 1;
      }
    } else if (threadIdx.x == 0) {
      // dependent column: its projections were accumulated into R; drop the remainder
    }
    __syncthreads();
  }
  if (qsh) {
    const int qc = s_qc;
    for (int e = threadIdx.x; e < s * qc; e += blockDim.x) F[e] = Fq[e];
  }
  if (threadIdx.x == 0) { qcols[u] = s_qc; qmode[u] = 0; }
}

// Recompression, step 2a: the cores C = R_a R_b^t (qa x qb, column-major, ld qa, at
// Cb + (a / 2) QCAP^2) of the sibling pairs a = list[blockIdx.y], one kCT x kCT tile of C
// per CTA (blockIdx.x).  Two kernels compute them: core_product_cc on CUDA cores (either
// precision) and, in complex64, core_product_tc on tensor cores; the setup times both on
// a layer of representative ranks and keeps the faster for each kind of recompression
// launch (factor_impl).
constexpr int kCT = 32;    // tile edge in complex entries
constexpr int kCK = 16;    // complex k chunk staged in shared memory

__device__ __forceinline__ bool core_tile(int qa, int qb, int tile, int& ti, int& tj) {
  const int ni = (qa + kCT - 1) / kCT, nj = (qb + kCT - 1) / kCT;
  if (tile >= ni * nj) return false;
  ti = tile % ni;
  tj = tile / ni;
  return true;
}

// 256 threads: thread (tx, ty) of a 16 x 16 grid owns rows ty, ty + 16 and columns tx,
// tx + 16 of the tile; the k chunks of R_a and R_b are staged with coalesced loads
template <typename R>
__global__ void __launch_bounds__(256) core_product_cc(Geo g, const Cx<R>* __restrict__ Rb,
                                                       const int* __restrict__ qcols, const int* __restrict__ G_rank,
                                                       Cx<R>* __restrict__ Cb) {
  __shared__ Cx<R> As[kCK][kCT + 1], Bs[kCK][kCT + 1];
  const int a = g.list[blockIdx.y], b = a + 1;
  const int qa = qcols[a], qb = qcols[b], w = G_rank[a];
  int ti, tj;
  if (!core_tile(qa, qb, blockIdx.x, ti, tj)) return;
  const Cx<R>* Ra = Rb + g.rbo[a];
  const Cx<R>* Rbb = Rb + g.rbo[b];
  const int lda = g.cap[a], ldb = g.cap[b];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  Cx<R> acc[2][2];
  for (int u = 0; u < 2; ++u)
    for (int v = 0; v < 2; ++v) acc[u][v] = Cx<R>(0, 0);
  for (int k0 = 0; k0 < w; k0 += kCK) {
    for (int e = threadIdx.x; e < kCK * kCT; e += blockDim.x) {
      const int kk = e % kCK, r = e / kCK;
      const int i = ti * kCT + r, j = tj * kCT + r, k = k0 + kk;
      As[kk][r] = (i < qa && k < w) ? Ra[(long long)i * lda + k] : Cx<R>(0, 0);
      Bs[kk][r] = (j < qb && k < w) ? Rbb[(long long)j * ldb + k] : Cx<R>(0, 0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kCK; ++kk) {
      const Cx<R> a0 = As[kk][ty], a1 = As[kk][ty + 16], b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      cfma(acc[0][0], a0, b0);
      cfma(acc[0][1], a0, b1);
      cfma(acc[1][0], a1, b0);
      cfma(acc[1][1], a1, b1);
    }
    __syncthreads();
  }
  Cx<R>* C = Cb + (long long)(a >> 1) * g.QCAP * g.QCAP;
  for (int u = 0; u < 2; ++u)
    for (int v = 0; v < 2; ++v) {
      const int i = ti * kCT + ty + 16 * u, j = tj * kCT + tx + 16 * v;
      if (i < qa && j < qb) C[(long long)j * qa + i] = acc[u][v];
    }
}

// x = hi + lo with hi the TF32 rounding of x (10 explicit mantissa bits) and lo = x - hi,
// exact in FP32; a product in three TF32 parts, hi*hi + hi*lo + lo*hi with FP32
// accumulation, keeps about 2^-21 relative accuracy
__device__ __forceinline__ void tf32_split(float x, unsigned& hi, unsigned& lo) {
  hi = (__float_as_uint(x) + 0x1000u) & 0xffffe000u;
  lo = __float_as_uint(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_m16n8k8_tf32(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
               : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The complex product as one real product C' = A' B'^t: A' row i = (Re, Im) of row i of
// R_a interleaved (real k' = 2 l + q), and B' holds for output column n' = 2 j + p
//   B'[2l][2j] = Re b, B'[2l+1][2j] = -Im b, B'[2l][2j+1] = Im b, B'[2l+1][2j+1] = Re b
// (b = R_b[j][l]), so that C'[i][2j] = Re C[i][j] and C'[i][2j+1] = Im C[i][j].  Eight
// warps: warp (wm = warp & 1, wn = warp >> 1) owns tile rows 16 wm .. 16 wm + 15 and the
// real columns 16 wn .. 16 wn + 15 (two m16n8k8 column tiles).
__global__ void __launch_bounds__(256) core_product_tc(Geo g, const Cx<float>* __restrict__ Rb,
                                                       const int* __restrict__ qcols, const int* __restrict__ G_rank,
                                                       Cx<float>* __restrict__ Cb) {
  __shared__ Cx<float> As[kCT][kCK + 1], Bs[kCT][kCK + 1];
  const int a = g.list[blockIdx.y], b = a + 1;
  const int qa = qcols[a], qb = qcols[b], w = G_rank[a];
  int ti, tj;
  if (!core_tile(qa, qb, blockIdx.x, ti, tj)) return;
  const Cx<float>* Ra = Rb + g.rbo[a];
  const Cx<float>* Rbb = Rb + g.rbo[b];
  const int lda = g.cap[a], ldb = g.cap[b];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wm = warp & 1, wn = warp >> 1;
  const int gid = lane >> 2, tig = lane & 3;
  float c[2][4] = {}, c2[2][4] = {};
  for (int k0 = 0; k0 < w; k0 += kCK) {
    for (int e = threadIdx.x; e < kCK * kCT; e += blockDim.x) {
      const int kk = e % kCK, r = e / kCK;
      const int i = ti * kCT + r, j = tj * kCT + r, k = k0 + kk;
      As[r][kk] = (i < qa && k < w) ? Ra[(long long)i * lda + k] : Cx<float>(0.f, 0.f);
      Bs[r][kk] = (j < qb && k < w) ? Rbb[(long long)j * ldb + k] : Cx<float>(0.f, 0.f);
    }
    __syncthreads();
    // real k' in steps of 8 over the chunk's 2 kCK real columns
#pragma unroll
    for (int ks = 0; ks < 2 * kCK; ks += 8) {
      // A fragment: rows 16 wm + gid (+ 8), real columns ks + tig (+ 4)
      unsigned ah[4], al[4];
      {
        const int r0 = 16 * wm + gid, r1 = r0 + 8;
        const int k1 = ks + tig, k2 = ks + tig + 4;
        const float v0 = (k1 & 1) ? As[r0][k1 >> 1].im : As[r0][k1 >> 1].re;
        const float v1 = (k1 & 1) ? As[r1][k1 >> 1].im : As[r1][k1 >> 1].re;
        const float v2 = (k2 & 1) ? As[r0][k2 >> 1].im : As[r0][k2 >> 1].re;
        const float v3 = (k2 & 1) ? As[r1][k2 >> 1].im : As[r1][k2 >> 1].re;
        tf32_split(v0, ah[0], al[0]);
        tf32_split(v1, ah[1], al[1]);
        tf32_split(v2, ah[2], al[2]);
        tf32_split(v3, ah[3], al[3]);
      }
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        // B fragment: real rows ks + tig (+ 4), real output column 16 wn + 8 nt + gid
        const int np = 16 * wn + 8 * nt + gid;
        const int j = np >> 1, p = np & 1;
        float bv[2];
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int kp = ks + tig + 4 * h2;
          const Cx<float> bb = Bs[j][kp >> 1];
          const int q = kp & 1;
          bv[h2] = p == 0 ? (q == 0 ? bb.re : -bb.im) : (q == 0 ? bb.im : bb.re);
        }
        unsigned bh0, bl0, bh1, bl1;
        tf32_split(bv[0], bh0, bl0);
        tf32_split(bv[1], bh1, bl1);
        mma_m16n8k8_tf32(c[nt], ah, bh0, bh1);
        mma_m16n8k8_tf32(c2[nt], al, bh0, bh1);
        mma_m16n8k8_tf32(c2[nt], ah, bl0, bl1);
      }
    }
    __syncthreads();
  }
  Cx<float>* C = Cb + (long long)(a >> 1) * g.QCAP * g.QCAP;
#pragma unroll
  for (int nt = 0; nt < 2; ++nt) {
    const int j = tj * kCT + ((16 * wn + 8 * nt) >> 1) + tig;   // output columns 2 tig, 2 tig + 1 of the n-tile
    const int i0 = ti * kCT + 16 * wm + gid, i1 = i0 + 8;
    if (j < qb) {
      if (i0 < qa) C[(long long)j * qa + i0] = Cx<float>(c[nt][0] + c2[nt][0], c[nt][1] + c2[nt][1]);
      if (i1 < qa) C[(long long)j * qa + i1] = Cx<float>(c[nt][2] + c2[nt][2], c[nt][3] + c2[nt][3]);
    }
  }
}

// Shuffle-sum within aligned groups of GW lanes (GW = 16 or 32).
template <typename R> __device__ __forceinline__ Cx<R> group_sum(Cx<R> v, int GW) {
  for (int o = GW >> 1; o > 0; o >>= 1) v += shfl_xor(v, o);
  return v;
}

// Recompression, step 2b: for every sibling pair (a, b) with a = list[blockIdx.x], the
// core C (step 2a), one-sided Jacobi C W = P Sigma, truncation, and the small transforms
//   T_a = (P Sigma)[:, kept] (qa x k'),  T_b = conj(W)[:, kept] (qb x k').
// qa, qb <= QCAP, the largest core of the plan (setup_alloc).
template <typename R>
__global__ void svd_jacobi(Geo g, double eps, const Cx<R>* __restrict__ Cb, const int* __restrict__ qcols,
                           const int* __restrict__ G_rank, Cx<R>* __restrict__ Wb, Cx<R>* __restrict__ Tx,
                           int* __restrict__ newrank, int smem_entries, R frz) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int a = g.list[blockIdx.x], b = a + 1, t = a >> 1;
  const int qa = qcols[a], qb = qcols[b];
  // C (column-major qa x qb, ld qa) and, when both fit in the shared-memory plan, the
  // accumulated rotations W (column-major qb x qb, ld qb); otherwise W stays in Wb
  const bool w_shared = (long long)qa * qb + (long long)qb * qb <= smem_entries;
  Cx<R>* C = reinterpret_cast<Cx<R>*>(sm);
  Cx<R>* Wm = w_shared ? C + (size_t)qa * qb : Wb + (long long)t * g.QCAP * g.QCAP;
  const int ldw = w_shared ? qb : g.QCAP;
  R* sig = reinterpret_cast<R*>(reinterpret_cast<Cx<R>*>(sm) + smem_entries);   // [QCAP + 1]
  int* order = reinterpret_cast<int*>(sig + g.QCAP + 1);                          // [QCAP]
  __shared__ int s_rot, s_keep;
  __shared__ R s_scale;
  if (qa == 0 || qb == 0) {
    if (threadIdx.x == 0) { newrank[a] = 0; newrank[b] = 0; }
    return;
  }
  {
    const Cx<R>* Cg = Cb + (long long)t * g.QCAP * g.QCAP;     // the core from step 2a
    for (int e = threadIdx.x; e < qa * qb; e += blockDim.x) C[e] = Cg[e];
  }
  for (int e = threadIdx.x; e < qb * qb; e += blockDim.x) {
    const int i = e % qb, j = e / qb;
    Wm[(long long)j * ldw + i] = Cx<R>(i == j ? 1 : 0, 0);
  }
  __syncthreads();
  // normalise by the largest column norm
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = warp; j < qb; j += nw) {
    R acc = 0;
    for (int i = lane; i < qa; i += 32) acc += abs2(C[(long long)j * qa + i]);
    acc = warp_sum_r(acc);
    if (lane == 0) sig[j] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    R mx = 0;
    for (int j = 0; j < qb; ++j) mx = fmax(mx, sig[j]);
    s_scale = sqrt(mx);
  }
  __syncthreads();
  const R scale = s_scale;
  if (!(scale > 0)) {
    if (threadIdx.x == 0) { newrank[a] = 0; newrank[b] = 0; }
    return;
  }
  const R iscale = R(1) / scale;
  for (int e = threadIdx.x; e < qa * qb; e += blockDim.x) C[e] = iscale * C[e];
  __syncthreads();
  const int me = qb + (qb & 1);               // even number of positions (one dummy if odd)
  // one group of GW lanes per column pair: whole warps while there are at most as many
  // pairs as warps, half warps beyond (every pair of a round in one pass)
  const int GW = (me / 2 <= nw) ? 32 : 16;
  const int gpw = 32 / GW;                    // groups per warp
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    // squared column norms, exact at the start of every sweep and carried through its
    // rounds by the rotation's own update (a rotation by tan t of the pair (p, q) with
    // <p, q> = g maps |p|^2 to |p|^2 - t |g| and |q|^2 to |q|^2 + t |g|), so a pair's test
    // needs only the inner product
    for (int j = warp; j < qb; j += nw) {
      R acc = 0;
      for (int i = lane; i < qa; i += 32) acc += abs2(C[(long long)j * qa + i]);
      acc = warp_sum_r(acc);
      if (lane == 0) sig[j] = acc;
    }
    __syncthreads();
    for (int round = 0; round < me - 1; ++round) {
      // the loop bound is uniform over the warp, so every lane reaches every shuffle
      for (int pb = warp * gpw; pb < me / 2; pb += nw * gpw) {
        const int pr = pb + lane / GW, gl = lane % GW;
        int p0 = pr, p1 = me - 1 - pr;
        int ip = p0 == 0 ? 0 : ((p0 - 1 + round) % (me - 1)) + 1;
        int iq = ((p1 - 1 + round) % (me - 1)) + 1;
        const bool live = pr < me / 2 && ip < qb && iq < qb;
        if (ip > iq) { int tmp = ip; ip = iq; iq = tmp; }
        Cx<R>* cp = C + (long long)(live ? ip : 0) * qa;
        Cx<R>* cq = C + (long long)(live ? iq : 0) * qa;
        const R al = live ? sig[ip] : R(0), be = live ? sig[iq] : R(0);
        Cx<R> ga(0, 0);
        if (live)
          for (int i = gl; i < qa; i += GW) cfma_conj(ga, cp[i], cq[i]);
        ga = group_sum(ga, GW);
        const R ag = sqrt(abs2(ga));
        // a column whose squared norm is below frz (relative to the largest, 1 after the
        // normalisation) stays below it under every rotation and is truncated in the end:
        // it is left alone, so the sweeps stop once the significant columns are orthogonal
        const bool rot = live && al >= frz && be >= frz && ag > Tiny<R>::jac * sqrt(al) * sqrt(be);
        if (rot) {
          if (gl == 0) s_rot = 1;
          const Cx<R> e(ga.re / ag, ga.im / ag);
          const R z = (be - al) / (R(2) * ag);
          const R tt = fabs(z) < R(1e18) ? (z >= 0 ? R(1) : R(-1)) / (fabs(z) + sqrt(R(1) + z * z)) : R(0.5) / z;
          const R cs = R(1) / sqrt(R(1) + tt * tt), sn = tt * cs;
          const Cx<R> snc = sn * conj(e), sne = sn * e;
          if (gl == 0) {
            sig[ip] = fmax(R(0), al - tt * ag);
            sig[iq] = be + tt * ag;
          }
          for (int i = gl; i < qa; i += GW) {
            const Cx<R> x = cp[i], y = cq[i];
            cp[i] = cs * x - snc * y;
            cq[i] = sne * x + cs * y;
          }
          Cx<R>* wp = Wm + (long long)ip * ldw;
          Cx<R>* wq = Wm + (long long)iq * ldw;
          for (int i = gl; i < qb; i += GW) {
            const Cx<R> x = wp[i], y = wq[i];
            wp[i] = cs * x - snc * y;
            wq[i] = sne * x + cs * y;
          }
        }
      }
      __syncthreads();
    }
    if (s_rot == 0) break;
    __syncthreads();
  }
  // singular values, ordering, truncation
  for (int j = warp; j < qb; j += nw) {
    R acc = 0;
    for (int i = lane; i < qa; i += 32) acc += abs2(C[(long long)j * qa + i]);
    acc = warp_sum_r(acc);
    if (lane == 0) sig[j] = sqrt(acc);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < qb; j += blockDim.x) {
    int rk = 0;
    for (int l = 0; l < qb; ++l) rk += (sig[l] > sig[j] || (sig[l] == sig[j] && l < j)) ? 1 : 0;
    order[rk] = j;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const R smax = sig[order[0]];
    int keep = 0;
    while (keep < qb && keep < g.r_max && smax > 0 && sig[order[keep]] > R(eps) * smax && sig[order[keep]] > 0) ++keep;
    s_keep = keep;
    newrank[a] = keep;
    newrank[b] = keep;
  }
  __syncthreads();
  const int keep = s_keep;
  Cx<R>* Ta = Tx + (long long)a * g.QCAP * g.r_max;   // column-major (ld QCAP)
  Cx<R>* Tb = Tx + (long long)b * g.QCAP * g.r_max;
  // balanced split: T_a = P_j sigma_j^(1/2), T_b = conj(W_j) sigma_j^(1/2)
  for (int e = threadIdx.x; e < qa * keep; e += blockDim.x) {
    const int i = e % qa, j = e / qa;
    const R f = sqrt(scale / sig[order[j]]);
    Ta[(long long)j * g.QCAP + i] = f * C[(long long)order[j] * qa + i];
  }
  for (int e = threadIdx.x; e < qb * keep; e += blockDim.x) {
    const int i = e % qb, j = e / qb;
    const R f = sqrt(scale * sig[order[j]]);
    Tb[(long long)j * g.QCAP + i] = f * conj(Wm[(long long)order[j] * ldw + i]);
  }
}

// Recompression, step 3, for the nodes u = list[blockIdx.y]: F'_u = Q_u T_u (sz(u) x kr,
// column-major; T_u itself on the dense path) into the node's region of the scratch
// buffer Fs, one kCT x kCT tile per CTA (blockIdx.x), the k chunks of Q_u and T_u staged
// with coalesced loads; recompress_copy then moves it into G_F (Q_u is read from G_F
// until every tile is done).
template <typename R>
__global__ void __launch_bounds__(256) recompress_gemm(Geo g, const Cx<R>* __restrict__ G_F,
                                                       const int* __restrict__ qcols, const int* __restrict__ qmode,
                                                       const Cx<R>* __restrict__ Tx, const int* __restrict__ newrank,
                                                       Cx<R>* __restrict__ Fs) {
  __shared__ Cx<R> Qs[kCK][kCT + 1], Ts[kCK][kCT + 1];
  const int u = g.list[blockIdx.y];
  const int s = g.sz[u], qc = qcols[u], kr = newrank[u];
  const int ni = (s + kCT - 1) / kCT, nj = (kr + kCT - 1) / kCT;
  if ((int)blockIdx.x >= ni * nj) return;
  const int ti = blockIdx.x % ni, tj = blockIdx.x / ni;
  const Cx<R>* Qu = G_F + g.gfo[u];
  const Cx<R>* T = Tx + (long long)u * g.QCAP * g.r_max;
  Cx<R>* S = Fs + g.gfo[u];
  if (qmode[u]) {
    for (int e = threadIdx.x; e < kCT * kCT; e += blockDim.x) {
      const int i = ti * kCT + e % kCT, j = tj * kCT + e / kCT;
      if (i < s && j < kr) S[(long long)j * s + i] = T[(long long)j * g.QCAP + i];
    }
    return;
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  Cx<R> acc[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) acc[a][b] = Cx<R>(0, 0);
  for (int k0 = 0; k0 < qc; k0 += kCK) {
    for (int e = threadIdx.x; e < kCK * kCT; e += blockDim.x) {
      const int r = e % kCT, kq = e / kCT;          // Q: consecutive threads, consecutive rows
      const int i = ti * kCT + r, k = k0 + kq;
      Qs[kq][r] = (i < s && k < qc) ? Qu[(long long)k * s + i] : Cx<R>(0, 0);
      const int kt = e % kCK, cc = e / kCK;         // T: consecutive threads, consecutive k
      const int j = tj * kCT + cc, k2 = k0 + kt;
      Ts[kt][cc] = (j < kr && k2 < qc) ? T[(long long)j * g.QCAP + k2] : Cx<R>(0, 0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kCK; ++kk) {
      const Cx<R> a0 = Qs[kk][ty], a1 = Qs[kk][ty + 16], b0 = Ts[kk][tx], b1 = Ts[kk][tx + 16];
      cfma(acc[0][0], a0, b0);
      cfma(acc[0][1], a0, b1);
      cfma(acc[1][0], a1, b0);
      cfma(acc[1][1], a1, b1);
    }
    __syncthreads();
  }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int i = ti * kCT + ty + 16 * a, j = tj * kCT + tx + 16 * b;
      if (i < s && j < kr) S[(long long)j * s + i] = acc[a][b];
    }
}

template <typename R>
__global__ void recompress_copy(Geo g, const Cx<R>* __restrict__ Fs, const int* __restrict__ newrank,
                                Cx<R>* __restrict__ G_F, int* __restrict__ G_rank) {
  const int u = g.list[blockIdx.x];
  const int s = g.sz[u], kr = newrank[u];
  const Cx<R>* S = Fs + g.gfo[u];
  Cx<R>* F = G_F + g.gfo[u];
  for (int e = threadIdx.x; e < s * kr; e += blockDim.x) F[e] = S[e];
  if (threadIdx.x == 0) G_rank[u] = kr;
}

// T~_m into the factor store (leaf padding zeroed, factors truncated to r_max columns).
template <typename R>
__global__ void store_layer(Geo g, const Cx<R>* __restrict__ G_leaf, const Cx<R>* __restrict__ G_F,
                            const int* __restrict__ G_rank, Cx<R>* __restrict__ dst, const long long* __restrict__ off,
                            int* __restrict__ rank_dst) {
  const int v = blockIdx.x;   // 0: leaves, v >= 2: factors
  if (v == 0) {
    const int lf = g.leaf;
    const long long tot = (long long)(1 << g.L) * lf * lf;
    for (long long e = threadIdx.x; e < tot; e += blockDim.x) {
      const int lam = (1 << g.L) + (int)(e / (lf * lf));
      const int r = (int)(e % (lf * lf));
      const int a = r % lf, b = r / lf, s = g.sz[lam];
      dst[e] = (a < s && b < s) ? G_leaf[e] : Cx<R>(0, 0);
    }
    if (threadIdx.x == 0) { rank_dst[0] = 0; rank_dst[1] = 0; }
    return;
  }
  if (v < 2) return;
  const int s = g.sz[v], r = G_rank[v];
  const Cx<R>* F = G_F + g.gfo[v];
  for (int e = threadIdx.x; e < s * r; e += blockDim.x) dst[off[v] + e] = F[e];
  if (threadIdx.x == 0) rank_dst[v] = r;
}

}  // namespace

// ---------------------------------------------------------------------------------------
struct SetupWork {
  int KCAP = 0, WCAP = 0, QCAP = 0;
  long long gfo_total = 0;   // entries of one G factor buffer
  std::vector<long long> sfo, gfo, qro, rbo;
  std::vector<int> rowleaf, cap;
  // node lists of the recompression launches: for depth step d, the nodes of the
  // non-deferred depths below d (big_nodes[d] .. big_nodes[d+1]) and their left siblings
  // (big_pairs), then the nodes of the deferred depths (small_*) and all nodes (all_*)
  std::vector<int> lists;
  std::vector<int> big_nodes_off, big_pairs_off;
  int small_nodes_off = 0, small_nodes = 0, small_pairs_off = 0, small_pairs = 0;
  int all_nodes_off = 0, all_nodes = 0, all_pairs_off = 0, all_pairs = 0;
  long long* d_sfo = nullptr;
  long long* d_gfo = nullptr;
  long long* d_qro = nullptr;
  long long* d_rbo = nullptr;
  int* d_rowleaf = nullptr;
  int* d_cap = nullptr;
  int* d_lists = nullptr;
  void *S_leaf = nullptr, *S_F = nullptr, *G_leaf = nullptr, *G_F = nullptr, *G_F2 = nullptr;
  void *Y = nullptr, *W = nullptr, *Qr = nullptr, *PQ = nullptr, *M = nullptr, *Rb = nullptr;
  void *Wb = nullptr, *Tx = nullptr, *Cb = nullptr;
  int *S_rank = nullptr, *G_rank = nullptr, *qcols = nullptr, *qmode = nullptr, *newrank = nullptr;
};

void hsw_setup_free(hsweep_s* h) {
  if (!h->sw) return;
  SetupWork* w = h->sw;
  void* ptrs[] = {w->d_sfo, w->d_gfo, w->d_qro, w->d_rbo, w->d_rowleaf, w->d_cap, w->d_lists, w->S_leaf, w->S_F,
                  w->G_leaf, w->G_F, w->G_F2, w->Y, w->W, w->Qr, w->PQ, w->M, w->Rb, w->Wb, w->Tx, w->Cb, w->S_rank,
                  w->G_rank, w->qcols, w->qmode, w->newrank};
  for (void* p : ptrs) hsw_release(h, p);
  delete w;
  h->sw = nullptr;
}

static int depth_of_host(int v) { int d = 0; while ((2 << d) <= v) ++d; return d; }

static int setup_alloc(hsweep_s* h) {
  SetupWork* w = new (std::nothrow) SetupWork();
  if (!w) return HSWEEP_ERR_OOM;
  h->sw = w;
  const size_t es = h->fac_elem();
  const int nn = h->nnodes, L = h->L;
  w->KCAP = h->r_max + 1;
  w->WCAP = h->r_max + w->KCAP;
  // A depth is deferred when the largest core its blocks can reach at the end of a layer,
  // min(rows, depth x KCAP) (every depth step above appends at most KCAP columns), fits the
  // Jacobi SVD's shared memory; its blocks are recompressed once per layer.  The other
  // depths are recompressed after every depth step (at most WCAP columns).
  const size_t smem_cap = 227 * 1024 - 4096;
  const int qlim = (int)std::sqrt((double)(smem_cap / es));
  auto deferred_core = [&](int d) { return std::min(h->tree.maxsz(d), d * w->KCAP); };
  auto small_depth = [&](int d) { return deferred_core(d) <= qlim; };
  w->QCAP = w->WCAP;
  for (int d = 1; d <= L; ++d)
    if (small_depth(d)) w->QCAP = std::max(w->QCAP, deferred_core(d));
  w->sfo.assign(nn, 0);
  w->gfo.assign(nn, 0);
  w->qro.assign(nn, 0);
  w->rbo.assign(nn, 0);
  w->cap.assign(nn, 0);
  long long so = 0, go = 0, qo = 0, ro = 0;
  for (int v = 2; v < nn; ++v) {
    const int d = depth_of_host(v), sv = h->tree.sz[v];
    const int cv = small_depth(d) ? d * w->KCAP : w->WCAP;
    w->cap[v] = cv;
    w->sfo[v] = so; so += (long long)sv * w->KCAP;
    w->gfo[v] = go; go += (long long)sv * cv;
    w->qro[v] = qo; qo += (long long)cv * w->KCAP;
    w->rbo[v] = ro; ro += (long long)std::min(sv, cv) * cv;
  }
  // recompression lists
  w->lists.clear();
  w->big_nodes_off.assign(L + 1, 0);
  w->big_pairs_off.assign(L + 1, 0);
  for (int d = 0; d < L; ++d) {
    w->big_nodes_off[d] = (int)w->lists.size();
    for (int v = 2; v < nn; ++v)
      if (depth_of_host(v) > d && !small_depth(depth_of_host(v))) w->lists.push_back(v);
  }
  w->big_nodes_off[L] = (int)w->lists.size();
  for (int d = 0; d < L; ++d) {
    w->big_pairs_off[d] = (int)w->lists.size();
    for (int v = 2; v < nn; v += 2)
      if (depth_of_host(v) > d && !small_depth(depth_of_host(v))) w->lists.push_back(v);
  }
  w->big_pairs_off[L] = (int)w->lists.size();
  w->small_nodes_off = (int)w->lists.size();
  for (int v = 2; v < nn; ++v)
    if (small_depth(depth_of_host(v))) w->lists.push_back(v);
  w->small_nodes = (int)w->lists.size() - w->small_nodes_off;
  w->small_pairs_off = (int)w->lists.size();
  for (int v = 2; v < nn; v += 2)
    if (small_depth(depth_of_host(v))) w->lists.push_back(v);
  w->small_pairs = (int)w->lists.size() - w->small_pairs_off;
  w->all_nodes_off = (int)w->lists.size();
  for (int v = 2; v < nn; ++v) w->lists.push_back(v);
  w->all_nodes = nn - 2;
  w->all_pairs_off = (int)w->lists.size();
  for (int v = 2; v < nn; v += 2) w->lists.push_back(v);
  w->all_pairs = (nn - 2) / 2;

  w->rowleaf.assign(h->n, 0);
  for (int lam = h->nleaves; lam < 2 * h->nleaves; ++lam)
    for (int i = 0; i < h->tree.sz[lam]; ++i) w->rowleaf[h->tree.lo[lam] + i] = lam;
  const long long lf2 = (long long)h->nleaves * h->leaf * h->leaf;
  const long long ntau = std::max(1, h->nleaves / 2);
  int rc;
#define A(p, bytes) do { rc = hsw_alloc(h, (void**)&(p), (size_t)(bytes)); if (rc) return rc; } while (0)
  A(w->d_sfo, nn * sizeof(long long));
  A(w->d_gfo, nn * sizeof(long long));
  A(w->d_qro, nn * sizeof(long long));
  A(w->d_rbo, nn * sizeof(long long));
  A(w->d_rowleaf, h->n * sizeof(int));
  A(w->d_cap, nn * sizeof(int));
  A(w->d_lists, std::max<size_t>(1, w->lists.size()) * sizeof(int));
  A(w->S_leaf, lf2 * es);
  A(w->G_leaf, lf2 * es);
  A(w->S_F, std::max(so, 1LL) * es);
  A(w->G_F, std::max(go, 1LL) * es);
  A(w->G_F2, std::max(go, 1LL) * es);
  w->gfo_total = std::max(go, 1LL);
  A(w->Y, (long long)h->n * w->KCAP * es);
  A(w->W, (long long)h->n * w->KCAP * es);
  A(w->Qr, std::max(qo, 1LL) * es);
  A(w->PQ, ntau * 2 * w->KCAP * w->KCAP * es);
  A(w->M, ntau * 4 * w->KCAP * w->KCAP * es);
  A(w->Rb, std::max(ro, 1LL) * es);
  A(w->Wb, (long long)nn * w->QCAP * w->QCAP * es);
  A(w->Tx, (long long)nn * w->QCAP * h->r_max * es);
  A(w->Cb, (long long)(nn / 2) * w->QCAP * w->QCAP * es);
  A(w->S_rank, nn * sizeof(int));
  A(w->G_rank, nn * sizeof(int));
  A(w->qcols, nn * sizeof(int));
  A(w->qmode, nn * sizeof(int));
  A(w->newrank, nn * sizeof(int));
#undef A
  HSW_CUDA(cudaMemcpyAsync(w->d_sfo, w->sfo.data(), nn * sizeof(long long), cudaMemcpyHostToDevice, h->stream));
  HSW_CUDA(cudaMemcpyAsync(w->d_gfo, w->gfo.data(), nn * sizeof(long long), cudaMemcpyHostToDevice, h->stream));
  HSW_CUDA(cudaMemcpyAsync(w->d_qro, w->qro.data(), nn * sizeof(long long), cudaMemcpyHostToDevice, h->stream));
  HSW_CUDA(cudaMemcpyAsync(w->d_rbo, w->rbo.data(), nn * sizeof(long long), cudaMemcpyHostToDevice, h->stream));
  HSW_CUDA(cudaMemcpyAsync(w->d_cap, w->cap.data(), nn * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  HSW_CUDA(cudaMemcpyAsync(w->d_rowleaf, w->rowleaf.data(), h->n * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  if (!w->lists.empty())
    HSW_CUDA(cudaMemcpyAsync(w->d_lists, w->lists.data(), w->lists.size() * sizeof(int), cudaMemcpyHostToDevice,
                             h->stream));
  HSW_CUDA(cudaMemsetAsync(w->S_rank, 0, nn * sizeof(int), h->stream));
  // the host vectors above are read by the asynchronous copies: keep them until the copies ran
  HSW_CUDA(cudaStreamSynchronize(h->stream));
  return HSWEEP_OK;
}

template <typename R>
static int factor_impl(hsweep_s* h) {
  SetupWork* w = h->sw;
  const size_t es = sizeof(Cx<R>);
  Geo g;
  g.n = h->n; g.L = h->L; g.leaf = h->leaf; g.nnodes = h->nnodes; g.r_max = h->r_max;
  g.KCAP = w->KCAP; g.WCAP = w->WCAP; g.QCAP = w->QCAP;
  g.lo = h->d_lo; g.sz = h->d_sz; g.rowleaf = w->d_rowleaf; g.sfo = w->d_sfo; g.gfo = w->d_gfo;
  g.cap = w->d_cap; g.qro = w->d_qro; g.rbo = w->d_rbo; g.list = w->d_lists;
  cudaStream_t st = h->stream;
  Cx<R>* fac = reinterpret_cast<Cx<R>*>(h->d_fac);
  Cx<R>* S_leaf = (Cx<R>*)w->S_leaf;
  Cx<R>* S_F = (Cx<R>*)w->S_F;
  Cx<R>* G_leaf = (Cx<R>*)w->G_leaf;
  Cx<R>* G_F = (Cx<R>*)w->G_F;
  Cx<R>* G_F2 = (Cx<R>*)w->G_F2;
  Cx<R>* Y = (Cx<R>*)w->Y;
  Cx<R>* Wv = (Cx<R>*)w->W;
  Cx<R>* Qr = (Cx<R>*)w->Qr;
  Cx<R>* PQ = (Cx<R>*)w->PQ;
  Cx<R>* M = (Cx<R>*)w->M;
  Cx<R>* Rb = (Cx<R>*)w->Rb;
  Cx<R>* Wb = (Cx<R>*)w->Wb;
  Cx<R>* Tx = (Cx<R>*)w->Tx;
  const int L = h->L, nn = h->nnodes, KCAP = w->KCAP, QCAP = w->QCAP;
  const size_t core_smem = (size_t)(2 * KCAP) * (2 * KCAP) * es + 32 * sizeof(R) + (2 * KCAP + 1) * sizeof(int) + 16;
  // QR: v, c and the reduction scratch, then as many entries of F_u as fit (226 KB in all)
  const size_t qr_base = ((size_t)(h->tree.maxsz(1) + QCAP) * es + 32 * sizeof(R) + 15) & ~size_t(15);
  const int qs_entries = qr_base < 226 * 1024 ? (int)((226 * 1024 - qr_base) / es) : 0;
  const size_t qr_smem = qr_base + (size_t)qs_entries * es;
  // the Jacobi SVD's shared memory: C and, where it fits, the rotations W (up to 2 QCAP^2
  // entries; for large cores W stays in global memory)
  const size_t svd_tail = (size_t)(QCAP + 1) * sizeof(R) + (size_t)QCAP * sizeof(int) + 64;
  // (1 KB of the 227 KB per block stays free for the kernel's static shared variables)
  const int svd_entries = (int)std::min<size_t>((size_t)2 * QCAP * QCAP, (226 * 1024 - svd_tail) / es);
  const size_t svd_smem = (size_t)svd_entries * es + svd_tail;
  // one shared-memory carveout for every kernel of the layer loop, so that consecutive
  // launches do not reconfigure the SMs' L1/shared split
  {
    const void* ks[] = {(const void*)schur_leaves<R>, (const void*)schur_factors<R>, (const void*)leaf_inverse<R>,
                        (const void*)tsmm_reduce<R>, (const void*)tsmm_expand<R>, (const void*)core_dots<R>,
                        (const void*)core_inverse<R>, (const void*)woodbury_form<R>, (const void*)woodbury_append<R>,
                        (const void*)qr_cgs2<R>, (const void*)svd_jacobi<R>, (const void*)recompress_gemm<R>,
                        (const void*)recompress_copy<R>, (const void*)store_layer<R>, (const void*)core_product_cc<R>};
    for (const void* k : ks)
      HSW_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared));
  }
  HSW_CUDA(cudaFuncSetAttribute(core_inverse<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)core_smem));
  HSW_CUDA(cudaFuncSetAttribute(qr_cgs2<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qr_smem));
  HSW_CUDA(cudaFuncSetAttribute(svd_jacobi<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)svd_smem));
  if (core_smem > 227 * 1024 || qr_smem > 227 * 1024 || svd_smem > 227 * 1024 || svd_entries < QCAP * QCAP)
    return HSWEEP_ERR_ARG;

  // Autotuning of the core products (step 2a), complex64 only: on layer tune_m, the first
  // launch of each kind (0: the recompressions after a depth step, 1: the once-per-layer
  // recompression) runs both kernels, timed with CUDA events, and the faster one serves that
  // kind of launch from then on; before it, and in complex128, the CUDA-core kernel runs.
  const int tune_m = h->n / 2;
  // Jacobi: columns below a tenth of the truncation threshold (squared, relative) are frozen
  const R frz = (R)std::max((double)Tiny<R>::neg, 0.01 * h->eps_H * h->eps_H);
  const int core_tiles = ((QCAP + kCT - 1) / kCT) * ((QCAP + kCT - 1) / kCT);
  const int gemm_tiles = ((h->tree.maxsz(1) + kCT - 1) / kCT) * ((h->r_max + kCT - 1) / kCT);
  Cx<R>* Cb = (Cx<R>*)w->Cb;
  int m_cur = 0;
  auto core_product = [&](const Geo& gp, int np_list, int kind) -> int {
    const dim3 grid(core_tiles, np_list);
    const bool f32 = sizeof(R) == 4;
    auto run = [&](int mode) {
      if constexpr (sizeof(R) == 4) {
        if (mode == 1) {
          core_product_tc<<<grid, 256, 0, st>>>(gp, (const Cx<float>*)Rb, w->qcols, w->G_rank, (Cx<float>*)Cb);
          return;
        }
      }
      core_product_cc<R><<<grid, 256, 0, st>>>(gp, Rb, w->qcols, w->G_rank, Cb);
    };
    if (h->opt.core_kernel > 0) {          // fixed by the caller
      run(f32 && h->opt.core_kernel == 2 ? 1 : 0);
      h->nlaunch += 1;
      return HSWEEP_OK;
    }
    if (f32 && h->core_mode[kind] < 0 && m_cur == tune_m) {
      cudaEvent_t ev[3];
      for (auto& e : ev) HSW_CUDA(cudaEventCreate(&e));
      HSW_CUDA(cudaEventRecord(ev[0], st));
      run(0);
      HSW_CUDA(cudaEventRecord(ev[1], st));
      run(1);
      HSW_CUDA(cudaEventRecord(ev[2], st));
      HSW_CUDA(cudaEventSynchronize(ev[2]));
      float t0 = 0, t1 = 0;
      HSW_CUDA(cudaEventElapsedTime(&t0, ev[0], ev[1]));
      HSW_CUDA(cudaEventElapsedTime(&t1, ev[1], ev[2]));
      for (auto& e : ev) cudaEventDestroy(e);
      h->core_ms[kind][0] = t0;
      h->core_ms[kind][1] = t1;
      h->core_mode[kind] = t1 < t0 ? 1 : 0;
      h->nlaunch += 2;
      return HSWEEP_OK;
    }
    run(f32 && h->core_mode[kind] == 1 ? 1 : 0);
    h->nlaunch += 1;
    return HSWEEP_OK;
  };

  // QR (or the dense path), the cores, their SVD and the new factors, for nn_list nodes
  // whose list starts at node_off and their np_list left siblings at pair_off
  auto recompress = [&](int node_off, int nn_list, int pair_off, int np_list, int kind) -> int {
    if (nn_list <= 0) return HSWEEP_OK;
    Geo gl = g;
    gl.list = w->d_lists + node_off;
    qr_cgs2<R><<<nn_list, 1024, qr_smem, st>>>(gl, G_F, w->G_rank, Rb, w->qcols, w->qmode, qs_entries);
    Geo gp = g;
    gp.list = w->d_lists + pair_off;
    int rc = core_product(gp, np_list, kind);
    if (rc) return rc;
    svd_jacobi<R><<<np_list, 1024, svd_smem, st>>>(gp, h->eps_H, Cb, w->qcols, w->G_rank, Wb, Tx, w->newrank,
                                                   svd_entries, frz);
    recompress_gemm<R><<<dim3(gemm_tiles, nn_list), 256, 0, st>>>(gl, G_F, w->qcols, w->qmode, Tx, w->newrank, G_F2);
    recompress_copy<R><<<nn_list, kBlk, 0, st>>>(gl, G_F2, w->newrank, G_F, w->G_rank);
    h->nlaunch += 4;
    return HSWEEP_OK;
  };

  for (int m = 0; m < h->n; ++m) {
    NvtxRange range("setup layer");
    m_cur = m;
    const Cx<R>* Tprev = m > 0 ? fac + (long long)(m - 1) * h->layer_stride : nullptr;
    const int* rprev = m > 0 ? h->d_rank + (long long)(m - 1) * nn : nullptr;
    schur_leaves<R><<<h->nleaves, 64, 0, st>>>(g, m, h->d_diag_m, h->d_east_m, h->d_north_m, Tprev, S_leaf);
    h->nlaunch += 1;
    if (nn > 2) {
      schur_factors<R><<<nn - 2, kBlk, 0, st>>>(g, m, h->d_east_m, h->d_north_m, Tprev, h->d_off, rprev, S_F,
                                                 w->S_rank);
      h->nlaunch += 1;
    }
    HSW_CUDA(cudaMemsetAsync(w->G_rank, 0, nn * sizeof(int), st));
    leaf_inverse<R><<<h->nleaves, 128, 0, st>>>(g, m, S_leaf, G_leaf, h->d_status);
    h->nlaunch += 1;
    for (int d = L - 1; d >= 0; --d) {
      const int n_below2 = (d + 2 <= L) ? (1 << (L + 1)) - (1 << (d + 2)) : 0;
      const int n_below1 = (1 << (L + 1)) - (1 << (d + 1));
      const int ntau_d = 1 << d;
      if (n_below2 > 0) {
        tsmm_reduce<R><<<n_below2, kBlk, 0, st>>>(g, d, G_F, w->G_rank, S_F, w->S_rank, Qr);
        h->nlaunch += 1;
      }
      tsmm_expand<R><<<dim3(div_up(h->n, 128), KCAP), 128, 0, st>>>(g, d, G_leaf, G_F, w->G_rank, S_F,
                                                                     w->S_rank, Qr, Y);
      h->nlaunch += 1;
      core_dots<R><<<dim3(2 * ntau_d, 8), kBlk, 0, st>>>(g, d, S_F, w->S_rank, Y, PQ);
      h->nlaunch += 1;
      core_inverse<R><<<ntau_d, 1024, core_smem, st>>>(g, d, m, w->S_rank, PQ, M, h->d_status);
      h->nlaunch += 1;
      woodbury_form<R><<<dim3(div_up(h->n, 128), KCAP), 128, 0, st>>>(g, d, w->S_rank, Y, M, Wv, G_F, w->G_rank);
      h->nlaunch += 1;
      woodbury_append<R><<<n_below1, kBlk, 0, st>>>(g, d, w->S_rank, Y, Wv, G_F, w->G_rank, G_leaf);
      h->nlaunch += 1;
      // the blocks of the non-deferred depths that this depth step changed
      int rc = recompress(w->big_nodes_off[d], w->big_nodes_off[d + 1] - w->big_nodes_off[d], w->big_pairs_off[d],
                          w->big_pairs_off[d + 1] - w->big_pairs_off[d], 0);
      if (rc) return rc;
    }
    // the blocks of the deferred depths, once per layer, in their final form
    {
      int rc = recompress(w->small_nodes_off, w->small_nodes, w->small_pairs_off, w->small_pairs, 1);
      if (rc) return rc;
    }
    if (h->strong_R > 0) {
      // strongly admissible T~_m (strong.cu), then one recompression of every sibling pair:
      // the expanded layout can carry more columns than a block has rows (small blocks,
      // blocks of rank below R); the recompression keeps the same matrix up to eps_H and
      // brings every rank to at most the block's dimensions, as the sweeps expect
      int rc = hsw_strong_project(h, m, G_F, w->G_rank, G_F2, w->d_gfo, w->gfo_total);
      if (rc) return rc;
      std::swap(G_F, G_F2);
      // the records of the strong sweep, from the exact strongly admissible factors
      rc = hsw_spack_layer(h, m, G_F, G_leaf, w->d_gfo);
      if (rc) return rc;
      rc = recompress(w->all_nodes_off, w->all_nodes, w->all_pairs_off, w->all_pairs, 1);
      if (rc) return rc;
    }
    store_layer<R><<<nn, kBlk, 0, st>>>(g, G_leaf, G_F, w->G_rank, fac + (long long)m * h->layer_stride,
                                        h->d_off, h->d_rank + (long long)m * nn);
    h->nlaunch += 1;
    HSW_CUDA(cudaGetLastError());
  }
  w->G_F = G_F;
  w->G_F2 = G_F2;
  return HSWEEP_OK;
}

int hsw_factor(hsweep_s* h) {
  if (!h->sw) {
    int rc = setup_alloc(h);
    if (rc) return rc;
  }
  if (h->prec == HSWEEP_FP64) return factor_impl<double>(h);
  return factor_impl<float>(h);
}
