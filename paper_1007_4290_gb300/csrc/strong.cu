// Strong admissibility (Section 2.3, the strongly admissible case).  Clusters i, i' of one
// depth are well separated when the distance between them is at least their width, on
// the bisection tree of a layer: |i - i'| >= 2.  A strongly admissible H-matrix keeps the
// blocks of the interaction lists (well separated, parents not) in factorised form of
// rank at most R, and the neighbouring leaves (the near field) densely.
//
// The GPU builds T~_m in strong form from the weakly admissible inverse of the setup
// (setup.cu), in two exact-layout steps per layer:
//   projection: every well-separated block (u, w) lies inside one sibling block (a, b) of
//     the weak form, S(u, w) = F_a[rows u] F_b[rows w]^t; its rank-R approximation comes
//     from the randomized SVD (Halko, Martinsson and Tropp; the paper uses it for
//     F = H . H): Y = S Omega with P = R + 8 Gaussian test vectors, Q = orth(Y),
//     B = Q^* S, and the dominant R-dimensional left singular subspace of B (Hermitian
//     Jacobi on B B^*) gives S ~ (Q V) (V^* B).  The near-field blocks (neighbouring
//     leaves) are formed densely;
//   expansion: the strong matrix is written back into the sibling-pair factor store
//     without approximation.  Inside a sibling block (a, b) the well-separated blocks
//     are, for every depth l below a, the three children (2c_a, 2c_b), (2c_a, 2c_b+1),
//     (2c_a+1, 2c_b+1) of the corner pair (c_a, c_b) (rightmost descendant of a, leftmost
//     of b at depth l-1), and the corner pair of leaves is dense, so F_a, F_b get the
//     columns [R per block | the corner block against the identity]: rank
//     3 R (L - depth(a)) + leaf.
// The next layer's S~_{m+1} and the sweeps read the expanded store, so both use the
// strongly admissible T~_m exactly.
#include <algorithm>
#include <cmath>
#include <vector>
#include "handle.h"

namespace {

constexpr int kThreads = 256;
constexpr int kOversample = 8;
constexpr int kPMax = 16;     // test vectors per block (R <= 8)
constexpr int kKMax = 56;     // rank of a weak block (r_max <= 56)

// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as
// 1, 2, 3", SC 2011): ten rounds of the multiply-xor bijection keyed by a Weyl sequence.
__host__ __device__ inline void philox_round(uint32_t c[4], const uint32_t k[2]) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  const uint32_t n0 = hi1 ^ c[1] ^ k[0], n2 = hi0 ^ c[3] ^ k[1];
  c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
}

}  // namespace

__host__ __device__ void hsw_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
    philox_round(c, k);
  }
  for (int i = 0; i < 4; ++i) out[i] = c[i];
}

namespace {

// Two complex standard normals (real and imaginary parts independent N(0, 1)) from one
// Philox block, by the Box-Muller transform.
template <typename R>
__device__ inline void gauss2(uint32_t row, uint32_t pair, uint32_t blk, uint32_t m, uint32_t seed, Cx<R>& z0,
                              Cx<R>& z1) {
  const uint32_t ctr[4] = {row, pair, blk, m};
  const uint32_t key[2] = {seed, 0x5EEDu};
  uint32_t x[4];
  hsw_philox4x32_10(ctr, key, x);
  const double s = 2.3283064365386963e-10;   // 2^-32
  const double u0 = ((double)x[0] + 0.5) * s, u1 = (double)x[1] * s;
  const double u2 = ((double)x[2] + 0.5) * s, u3 = (double)x[3] * s;
  const double r0 = sqrt(-2.0 * log(u0)), r1 = sqrt(-2.0 * log(u2));
  double s0, c0, s1, c1;
  sincospi(2.0 * u1, &s0, &c0);
  sincospi(2.0 * u3, &s1, &c1);
  z0 = Cx<R>(R(r0 * c0), R(r0 * s0));
  z1 = Cx<R>(R(r1 * c1), R(r1 * s1));
}

struct FarArgs {
  int nblk, R, P;
  uint32_t seed;
  const int* info;          // [nblk][8]: a, b, ru0, rw0, su, sw, col, depth of (u, w)
  const long long* soff;    // [nblk] scratch offset (entries): Omega/Bt (sw x P), then Y/Q (su x P)
  const long long* gfo;     // factor offsets per node
  const int* sz;            // node sizes
};

template <typename R>
__device__ inline R block_sum(R v, R* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  R t = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}

// One CTA per well-separated block: randomized rank-R projection, written into the
// expanded factors of the sibling pair (a, b) that contains it.
template <typename R>
__global__ void __launch_bounds__(kThreads) strong_far(FarArgs fa, int m, double eps, const Cx<R>* __restrict__ F,
                                                       const int* __restrict__ rank, Cx<R>* __restrict__ Fout,
                                                       Cx<R>* __restrict__ scratch) {
  __shared__ Cx<R> Z[kKMax * kPMax];
  __shared__ double Gre[kPMax * kPMax], Gim[kPMax * kPMax];
  __shared__ double Vre[kPMax * kPMax], Vim[kPMax * kPMax];
  __shared__ double lam[kPMax], scl[kPMax];
  __shared__ int order[kPMax];
  __shared__ Cx<R> coef[kPMax];
  __shared__ R red[32];
  __shared__ int s_q, s_keep;

  const int bi = blockIdx.x;
  const int* inf = fa.info + 8 * bi;
  const int a = inf[0], b = inf[1], ru0 = inf[2], rw0 = inf[3], su = inf[4], sw = inf[5], col = inf[6];
  const int k = rank[a];
  if (k <= 0) return;
  const int P = fa.P, tid = threadIdx.x;
  const int lda = fa.sz[a], ldb = fa.sz[b];
  const Cx<R>* Fa = F + fa.gfo[a] + ru0;
  const Cx<R>* Fb = F + fa.gfo[b] + rw0;
  Cx<R>* Om = scratch + fa.soff[bi];          // sw x P (Omega, later Bt), column-major
  Cx<R>* Y = Om + (long long)sw * P;          // su x P (Y, then Q), column-major

  // Omega: complex Gaussian test vectors
  for (int e = tid; e < sw * (P / 2); e += blockDim.x) {
    const int row = e % sw, pr = e / sw;
    Cx<R> z0, z1;
    gauss2<R>((uint32_t)row, (uint32_t)pr, (uint32_t)bi, (uint32_t)m, fa.seed, z0, z1);
    Om[(long long)(2 * pr) * sw + row] = z0;
    Om[(long long)(2 * pr + 1) * sw + row] = z1;
  }
  __syncthreads();
  // Z = F_b[rows w]^t Omega  (k x P)
  for (int e = tid; e < k * P; e += blockDim.x) {
    const int c = e % k, p = e / k;
    Cx<R> acc(0, 0);
    for (int r = 0; r < sw; ++r) cfma(acc, Fb[(long long)c * ldb + r], Om[(long long)p * sw + r]);
    Z[p * kKMax + c] = acc;
  }
  __syncthreads();
  // Y = F_a[rows u] Z  (su x P)
  for (int e = tid; e < su * P; e += blockDim.x) {
    const int r = e % su, p = e / su;
    Cx<R> acc(0, 0);
    for (int c = 0; c < k; ++c) cfma(acc, Fa[(long long)c * lda + r], Z[p * kKMax + c]);
    Y[(long long)p * su + r] = acc;
  }
  __syncthreads();
  // Q = orth(Y): classical Gram-Schmidt applied twice, dependent columns dropped
  const R keep_tol = sizeof(R) == 4 ? R(1e-5) : R(1e-12);
  if (tid == 0) s_q = 0;
  __syncthreads();
  for (int j = 0; j < P; ++j) {
    const int q = s_q;
    Cx<R>* y = Y + (long long)j * su;
    R n0 = 0;
    for (int r = tid; r < su; r += blockDim.x) n0 += abs2(y[r]);
    n0 = block_sum(n0, red);
    for (int pass = 0; pass < 2; ++pass) {
      for (int i = 0; i < q; ++i) {
        Cx<R> acc(0, 0);
        for (int r = tid; r < su; r += blockDim.x) cfma_conj(acc, Y[(long long)i * su + r], y[r]);
        const R re = block_sum(acc.re, red);
        const R im = block_sum(acc.im, red);
        if (tid == 0) coef[i] = Cx<R>(re, im);
      }
      __syncthreads();
      for (int r = tid; r < su; r += blockDim.x) {
        Cx<R> v = y[r];
        for (int i = 0; i < q; ++i) v -= coef[i] * Y[(long long)i * su + r];
        y[r] = v;
      }
      __syncthreads();
    }
    R n1 = 0;
    for (int r = tid; r < su; r += blockDim.x) n1 += abs2(y[r]);
    n1 = block_sum(n1, red);
    if (n1 > keep_tol * keep_tol * n0 && n1 > R(0)) {
      const R inv = R(1) / sqrt(n1);
      Cx<R>* dst = Y + (long long)q * su;
      for (int r = tid; r < su; r += blockDim.x) dst[r] = inv * y[r];
      __syncthreads();
      if (tid == 0) s_q = q + 1;
    }
    __syncthreads();
  }
  const int q = s_q;
  if (q == 0) return;
  // Z2 = F_a[rows u]^t conj(Q)  (k x q)
  for (int e = tid; e < k * q; e += blockDim.x) {
    const int c = e % k, p = e / k;
    Cx<R> acc(0, 0);
    for (int r = 0; r < su; ++r) cfma_conj(acc, Y[(long long)p * su + r], Fa[(long long)c * lda + r]);
    Z[p * kKMax + c] = acc;
  }
  __syncthreads();
  // Bt = F_b[rows w] Z2 = (Q^* S)^t  (sw x q), over Omega
  for (int e = tid; e < sw * q; e += blockDim.x) {
    const int r = e % sw, p = e / sw;
    Cx<R> acc(0, 0);
    for (int c = 0; c < k; ++c) cfma(acc, Fb[(long long)c * ldb + r], Z[p * kKMax + c]);
    Om[(long long)p * sw + r] = acc;
  }
  __syncthreads();
  // Gram matrix B B^* (q x q, Hermitian), FP64
  for (int e = tid; e < q * q; e += blockDim.x) {
    const int p = e % q, r = e / q;
    double re = 0, im = 0;
    for (int x = 0; x < sw; ++x) {
      const Cx<R> u = Om[(long long)p * sw + x], v = Om[(long long)r * sw + x];
      re += (double)u.re * v.re + (double)u.im * v.im;
      im += (double)u.im * v.re - (double)u.re * v.im;
    }
    Gre[p * kPMax + r] = re;
    Gim[p * kPMax + r] = im;
    Vre[p * kPMax + r] = p == r ? 1.0 : 0.0;
    Vim[p * kPMax + r] = 0.0;
  }
  __syncthreads();
  // cyclic Jacobi on the Hermitian Gram matrix, one warp: U = diag(1, e^{-i phi}) J with the
  // real symmetric Schur rotation J, G <- U^* G U, V <- V U
  if (tid < 32) {
    const int x = tid;
    for (int sweep = 0; sweep < 30; ++sweep) {
      double off = 0, dia = 0;
      for (int e = x; e < q * q; e += 32) {
        const int p = e % q, r = e / q;
        const double v2 = Gre[p * kPMax + r] * Gre[p * kPMax + r] + Gim[p * kPMax + r] * Gim[p * kPMax + r];
        if (p == r) dia += v2; else off += v2;
      }
      for (int o = 16; o; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        dia += __shfl_xor_sync(0xffffffffu, dia, o);
      }
      if (!(off > 1e-30 * dia)) break;
      for (int p = 0; p < q - 1; ++p)
        for (int r = p + 1; r < q; ++r) {
          const double gr = Gre[p * kPMax + r], gi = Gim[p * kPMax + r];
          const double ag = sqrt(gr * gr + gi * gi);
          const double ap = Gre[p * kPMax + p], ar = Gre[r * kPMax + r];
          if (!(ag > 1e-18 * sqrt(fabs(ap * ar)) && ag > 1e-300)) continue;
          const double tau = (ar - ap) / (2.0 * ag);
          const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
          const double er = gr / ag, ei = gi / ag;           // e^{i phi}
          __syncwarp();
          if (x < q) {     // columns p, r: col_p' = c col_p - s e^{-i phi} col_r, col_r' = s col_p + c e^{-i phi} col_r
            const double pr_ = Gre[x * kPMax + p], pi_ = Gim[x * kPMax + p];
            const double rr_ = Gre[x * kPMax + r], ri_ = Gim[x * kPMax + r];
            const double er_r = rr_ * er + ri_ * ei, er_i = ri_ * er - rr_ * ei;   // e^{-i phi} col_r
            Gre[x * kPMax + p] = c * pr_ - s * er_r; Gim[x * kPMax + p] = c * pi_ - s * er_i;
            Gre[x * kPMax + r] = s * pr_ + c * er_r; Gim[x * kPMax + r] = s * pi_ + c * er_i;
            const double vpr = Vre[x * kPMax + p], vpi = Vim[x * kPMax + p];
            const double vrr = Vre[x * kPMax + r], vri = Vim[x * kPMax + r];
            const double vr_r = vrr * er + vri * ei, vr_i = vri * er - vrr * ei;
            Vre[x * kPMax + p] = c * vpr - s * vr_r; Vim[x * kPMax + p] = c * vpi - s * vr_i;
            Vre[x * kPMax + r] = s * vpr + c * vr_r; Vim[x * kPMax + r] = s * vpi + c * vr_i;
          }
          __syncwarp();
          if (x < q) {     // rows p, r: row_p' = c row_p - s e^{i phi} row_r, row_r' = s row_p + c e^{i phi} row_r
            const double pr_ = Gre[p * kPMax + x], pi_ = Gim[p * kPMax + x];
            const double rr_ = Gre[r * kPMax + x], ri_ = Gim[r * kPMax + x];
            const double er_r = rr_ * er - ri_ * ei, er_i = ri_ * er + rr_ * ei;   // e^{i phi} row_r
            Gre[p * kPMax + x] = c * pr_ - s * er_r; Gim[p * kPMax + x] = c * pi_ - s * er_i;
            Gre[r * kPMax + x] = s * pr_ + c * er_r; Gim[r * kPMax + x] = s * pi_ + c * er_i;
          }
          __syncwarp();
        }
    }
    if (x == 0) {
      for (int p = 0; p < q; ++p) { lam[p] = Gre[p * kPMax + p]; order[p] = p; }
      for (int p = 1; p < q; ++p)
        for (int r = p; r > 0 && lam[order[r]] > lam[order[r - 1]]; --r) {
          const int t = order[r]; order[r] = order[r - 1]; order[r - 1] = t;
        }
      const double floor_rel = sizeof(R) == 4 ? 1e-12 : 1e-28;
      const double thr = lam[order[0]] * fmax(eps * eps, floor_rel);
      int keep = 0;
      while (keep < fa.R && keep < q && lam[order[keep]] > thr && lam[order[keep]] > 0) {
        scl[keep] = sqrt(sqrt(lam[order[keep]]));     // sigma^(1/2): balanced factors
        ++keep;
      }
      s_keep = keep;
    }
  }
  __syncthreads();
  const int keep = s_keep;
  // left = Q V[:, kept] sigma^(1/2) -> F'_a[rows u]; right = Bt conj(V[:, kept]) sigma^(-1/2) -> F'_b[rows w]
  Cx<R>* Oa = Fout + fa.gfo[a] + ru0;
  Cx<R>* Ob = Fout + fa.gfo[b] + rw0;
  for (int e = tid; e < su * keep; e += blockDim.x) {
    const int r = e % su, i = e / su, oi = order[i];
    double re = 0, im = 0;
    for (int p = 0; p < q; ++p) {
      const Cx<R> y = Y[(long long)p * su + r];
      const double vr = Vre[p * kPMax + oi], vi = Vim[p * kPMax + oi];
      re += y.re * vr - y.im * vi;
      im += y.re * vi + y.im * vr;
    }
    Oa[(long long)(col + i) * lda + r] = Cx<R>(R(re * scl[i]), R(im * scl[i]));
  }
  for (int e = tid; e < sw * keep; e += blockDim.x) {
    const int r = e % sw, i = e / sw, oi = order[i];
    double re = 0, im = 0;
    for (int p = 0; p < q; ++p) {
      const Cx<R> y = Om[(long long)p * sw + r];
      const double vr = Vre[p * kPMax + oi], vi = -Vim[p * kPMax + oi];
      re += y.re * vr - y.im * vi;
      im += y.re * vi + y.im * vr;
    }
    Ob[(long long)(col + i) * ldb + r] = Cx<R>(R(re / scl[i]), R(im / scl[i]));
  }
}

struct NearArgs {
  const int* info;          // [npairs][6]: a, b, ca0 (rows of c_a within a), na, nb, col
  const long long* gfo;
  const int* sz;
};

// One CTA per sibling pair (a, b): the dense near-field block of its corner leaves
// D = F_a[rows c_a] F_b[rows c_b]^t, written as the columns [D | I] of the expansion.
template <typename R>
__global__ void __launch_bounds__(128) strong_near(NearArgs na, const Cx<R>* __restrict__ F, const int* __restrict__ rank,
                                                   Cx<R>* __restrict__ Fout) {
  const int* inf = na.info + 6 * blockIdx.x;
  const int a = inf[0], b = inf[1], ca0 = inf[2], nA = inf[3], nB = inf[4], col = inf[5];
  const int k = rank[a];
  const int lda = na.sz[a], ldb = na.sz[b];
  const Cx<R>* Fa = F + na.gfo[a] + ca0;
  const Cx<R>* Fb = F + na.gfo[b];
  Cx<R>* Oa = Fout + na.gfo[a] + ca0;
  Cx<R>* Ob = Fout + na.gfo[b];
  for (int e = threadIdx.x; e < nA * nB; e += blockDim.x) {
    const int i = e % nA, c = e / nA;
    Cx<R> acc(0, 0);
    for (int t = 0; t < k; ++t) cfma(acc, Fa[(long long)t * lda + i], Fb[(long long)t * ldb + c]);
    Oa[(long long)(col + c) * lda + i] = acc;
  }
  for (int e = threadIdx.x; e < nB * nB; e += blockDim.x) {
    const int i = e % nB, c = e / nB;
    Ob[(long long)(col + c) * ldb + i] = Cx<R>(i == c ? R(1) : R(0), R(0));
  }
}

int depth_of_host(int v) { int d = 0; while (v > 1) { v >>= 1; ++d; } return d; }

}  // namespace

struct StrongWork {
  int nfar = 0, nnear = 0, P = 0;
  int* d_far = nullptr;
  long long* d_soff = nullptr;
  int* d_near = nullptr;
  int* d_rank = nullptr;        // expanded rank per node
  void* scratch = nullptr;
};

int hsw_strong_expansion_rank(int R, int L, int leaf) { return 3 * R * (L > 0 ? L - 1 : 0) + leaf; }

// The strong layout of one layer: far records {a, b, ru0, rw0, su, sw, col, l} (the block
// (u, w) of depth l inside the sibling pair (a, b), rows ru0.. of a and rw0.. of b, columns
// col..col+R of the expanded factors), near records {a, b, ca0, na, nb, col} (the corner
// leaves), and the expanded rank of every node.
static void strong_plan(const Tree& t, int R, std::vector<int>& far, std::vector<int>& near,
                        std::vector<int>& nrank) {
  const int L = t.L;
  far.clear(); near.clear();
  nrank.assign(t.nnodes, 0);
  // the sibling pairs (a, b) and, inside each, the corner chain down to the leaves
  for (int av = 2; av < t.nnodes; av += 2) {
    const int bv = av + 1, la = depth_of_host(av);
    int ca = av, cb = bv;      // corner pair at depth l - 1
    for (int l = la + 1; l <= L; ++l) {
      const int us[3] = {2 * ca, 2 * ca, 2 * ca + 1};
      const int ws[3] = {2 * cb, 2 * cb + 1, 2 * cb + 1};
      for (int tt = 0; tt < 3; ++tt) {
        const int u = us[tt], w = ws[tt];
        const int rec[8] = {av, bv, t.lo[u] - t.lo[av], t.lo[w] - t.lo[bv], t.sz[u], t.sz[w],
                            R * (3 * (l - la - 1) + tt), l};
        far.insert(far.end(), rec, rec + 8);
      }
      ca = 2 * ca + 1;
      cb = 2 * cb;
    }
    // ca, cb are now the corner leaves
    const int col = 3 * R * (L - la);
    const int rec[6] = {av, bv, t.lo[ca] - t.lo[av], t.sz[ca], t.sz[cb], col};
    near.insert(near.end(), rec, rec + 6);
    nrank[av] = nrank[bv] = col + t.sz[cb];
  }
}

static int strong_prepare(hsweep_s* h, size_t es) {
  StrongWork* s = new (std::nothrow) StrongWork();
  if (!s) return HSWEEP_ERR_OOM;
  h->stw = s;
  const Tree& t = h->tree;
  s->P = std::min(kPMax, (h->strong_R + kOversample + 1) / 2 * 2);
  std::vector<int> far, near, nrank;
  strong_plan(t, h->strong_R, far, near, nrank);
  for (int v = 2; v < h->nnodes; ++v)
    if (nrank[v] > h->r_max) return HSWEEP_ERR_ARG;
  std::vector<long long> soff;
  long long so = 0;
  for (size_t i = 0; i < far.size(); i += 8) {
    soff.push_back(so);
    so += (long long)(far[i + 4] + far[i + 5]) * s->P;
  }
  s->nfar = (int)soff.size();
  s->nnear = (int)(near.size() / 6);
  int rc;
  if ((rc = hsw_alloc(h, (void**)&s->d_far, std::max<size_t>(1, far.size()) * sizeof(int)))) return rc;
  if ((rc = hsw_alloc(h, (void**)&s->d_soff, std::max<size_t>(1, soff.size()) * sizeof(long long)))) return rc;
  if ((rc = hsw_alloc(h, (void**)&s->d_near, std::max<size_t>(1, near.size()) * sizeof(int)))) return rc;
  if ((rc = hsw_alloc(h, (void**)&s->d_rank, h->nnodes * sizeof(int)))) return rc;
  if ((rc = hsw_alloc(h, &s->scratch, (size_t)std::max(1LL, so) * es))) return rc;
  if (!far.empty())
    HSW_CUDA(cudaMemcpyAsync(s->d_far, far.data(), far.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  if (!soff.empty())
    HSW_CUDA(cudaMemcpyAsync(s->d_soff, soff.data(), soff.size() * sizeof(long long), cudaMemcpyHostToDevice, h->stream));
  if (!near.empty())
    HSW_CUDA(cudaMemcpyAsync(s->d_near, near.data(), near.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  HSW_CUDA(cudaMemcpyAsync(s->d_rank, nrank.data(), h->nnodes * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  // the host vectors go out of scope: wait for the copies
  HSW_CUDA(cudaStreamSynchronize(h->stream));
  return HSWEEP_OK;
}

void hsw_strong_free(hsweep_s* h) {
  if (!h->stw) return;
  StrongWork* s = h->stw;
  void* ptrs[] = {s->d_far, s->d_soff, s->d_near, s->d_rank, s->scratch};
  for (void* p : ptrs) hsw_release(h, p);
  delete s;
  h->stw = nullptr;
}

template <typename R>
static int project_impl(hsweep_s* h, int m, const Cx<R>* G_F, int* G_rank, Cx<R>* G_F2, const long long* d_gfo,
                        long long gf_entries) {
  if (!h->stw) {
    int rc = strong_prepare(h, sizeof(Cx<R>));
    if (rc) return rc;
  }
  StrongWork* s = h->stw;
  cudaStream_t st = h->stream;
  HSW_CUDA(cudaMemsetAsync(G_F2, 0, (size_t)gf_entries * sizeof(Cx<R>), st));
  if (s->nfar > 0) {
    FarArgs fa;
    fa.nblk = s->nfar; fa.R = h->strong_R; fa.P = s->P; fa.seed = h->opt.rsvd_seed;
    fa.info = s->d_far; fa.soff = s->d_soff; fa.gfo = d_gfo; fa.sz = h->d_sz;
    strong_far<R><<<s->nfar, kThreads, 0, st>>>(fa, m, h->eps_H, G_F, G_rank, G_F2, (Cx<R>*)s->scratch);
    h->nlaunch += 1;
  }
  if (s->nnear > 0) {
    NearArgs na;
    na.info = s->d_near; na.gfo = d_gfo; na.sz = h->d_sz;
    strong_near<R><<<s->nnear, 128, 0, st>>>(na, G_F, G_rank, G_F2);
    h->nlaunch += 1;
  }
  HSW_CUDA(cudaMemcpyAsync(G_rank, s->d_rank, h->nnodes * sizeof(int), cudaMemcpyDeviceToDevice, st));
  HSW_CUDA(cudaGetLastError());
  return HSWEEP_OK;
}

int hsw_strong_project(hsweep_s* h, int m, const void* G_F, int* G_rank, void* G_F2, const long long* d_gfo,
                       long long gf_entries) {
  if (h->prec == HSWEEP_FP64)
    return project_impl<double>(h, m, (const c128*)G_F, G_rank, (c128*)G_F2, d_gfo, gf_entries);
  return project_impl<float>(h, m, (const c64*)G_F, G_rank, (c64*)G_F2, d_gfo, gf_entries);
}

extern "C" int hsweep_strong_plan(int n, int leaf, int R, int* nfar, int* nnear, int* far, int* near, int* ranks) {
  if (n < 3 || n > 32767 || leaf < 2 || leaf > 8 || R < 1 || R > 8 || !nfar || !nnear) return HSWEEP_ERR_ARG;
  Tree t;
  t.build(n, leaf);
  std::vector<int> fv, nv, rk;
  strong_plan(t, R, fv, nv, rk);
  *nfar = (int)(fv.size() / 8);
  *nnear = (int)(nv.size() / 6);
  if (far) std::copy(fv.begin(), fv.end(), far);
  if (near) std::copy(nv.begin(), nv.end(), near);
  if (ranks) std::copy(rk.begin(), rk.end(), ranks);
  return HSWEEP_OK;
}

extern "C" int hsweep_rsvd_normals(uint32_t blk, uint32_t m, uint32_t seed, int rows, int P, double* out) {
  if (rows < 0 || P < 2 || (P & 1) || (rows > 0 && !out)) return HSWEEP_ERR_ARG;
  const double s = 2.3283064365386963e-10, two_pi = 6.283185307179586476925286766559;
  for (int pr = 0; pr < P / 2; ++pr)
    for (int row = 0; row < rows; ++row) {
      const uint32_t ctr[4] = {(uint32_t)row, (uint32_t)pr, blk, m};
      const uint32_t key[2] = {seed, 0x5EEDu};
      uint32_t x[4];
      hsw_philox4x32_10(ctr, key, x);
      const double u0 = ((double)x[0] + 0.5) * s, u1 = (double)x[1] * s;
      const double u2 = ((double)x[2] + 0.5) * s, u3 = (double)x[3] * s;
      const double r0 = std::sqrt(-2.0 * std::log(u0)), r1 = std::sqrt(-2.0 * std::log(u2));
      double* z0 = out + 2 * ((long long)(2 * pr) * rows + row);
      double* z1 = out + 2 * ((long long)(2 * pr + 1) * rows + row);
      z0[0] = r0 * std::cos(two_pi * u1); z0[1] = r0 * std::sin(two_pi * u1);
      z1[0] = r1 * std::cos(two_pi * u3); z1[1] = r1 * std::sin(two_pi * u3);
    }
  return HSWEEP_OK;
}

extern "C" int hsweep_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  if (!ctr || !key || !out) return HSWEEP_ERR_ARG;
  hsw_philox4x32_10(ctr, key, out);
  return HSWEEP_OK;
}
