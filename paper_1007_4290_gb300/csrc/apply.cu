// The apply z = M r of Algorithm 2.6: a forward sweep w_m = hmatvec(T~_m, u_m),
// u_{m+1} = f_{m+1} - A_{m+1,m} w_m (m = 1..n), the reuse u_n = w_n of the middle loop,
// and a backward sweep u_m = w_m - hmatvec(T~_m, A_{m,m+1} u_{m+1}) (m = n-1..1).
//
// One persistent kernel runs all 2n-1 dependent H-matrix-vector products (Section 2.3,
// "Matrix-vector multiplication").  A sweep TEAM of C = 2^dC CTAs carries a group of G
// right-hand sides through the whole sweep; CTA c of the team owns the rows of the
// tree node at depth dC with index c (its "slab").  Within a layer:
//   1. reductions q_v = F_v^t x_v for every node v meeting the slab (weakly admissible,
//      symmetric storage: the block (a, b) of siblings is F_a F_b^t);  nodes inside
//      the slab are summed in shared memory, the dC ancestors of the slab leave one
//      partial sum per CTA in an L2 exchange buffer (double-buffered by layer parity);
//   2. one team barrier (a hardware cluster barrier when the team is a thread-block
//      cluster; a bounded-spin grid barrier when the team is the whole grid);
//   3. each row i gets y_i = (D_leaf x)_i + sum over its L enclosing nodes v of
//      F_v[i, :] q_sibling(v), then the sweep update of Algorithm 2.6.
// The factors of a layer are read once per team and step (coalesced, column-major),
// every other quantity lives in shared memory.
#include <cooperative_groups.h>
#include "handle.h"

namespace cg = cooperative_groups;

namespace {

constexpr int kThreads = 512;
constexpr long long kSpinLimit = 4000000;   // bounded grid-barrier wait (about a second)

template <typename R>
struct SweepArgs {
  int n, L, leaf, r_max, nnodes, dC, C, nteams, nrhs, ngroups, slab_max;
  long long N, layer_stride;
  const int* lo;
  const int* sz;
  const long long* off;
  const Cx<R>* fac;
  const int* rank;
  const c128* north;
  const c128* r;
  c128* z;
  Cx<R>* w;
  Cx<R>* xch;
  int* status;
  unsigned* bar;
};

__device__ __forceinline__ int pow2ceil32(int x) {
  int g = 1;
  while (g < x && g < 32) g <<= 1;
  return g;
}

// Bounded-spin barrier over the whole (co-resident, cooperative) grid.  Returns false
// after recording HSWEEP_ERR_TIMEOUT when the wait runs out, or when another CTA
// already recorded an error.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, int* status, int layer) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = bar + 1;
    unsigned gen = *vgen;
    __threadfence();
    unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*vgen == gen) {
        if (++spins > kSpinLimit) { ok = 0; report_error(status, HSWEEP_ERR_TIMEOUT, layer); break; }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*(volatile int*)status != 0) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

template <typename R, int G, bool GRID>
__global__ void __launch_bounds__(kThreads, 1) sweep_kernel(SweepArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x;
  const int C = a.C, dC = a.dC, L = a.L, n = a.n, G_ = G;
  const int c = GRID ? blockIdx.x : (int)cg::this_cluster().block_rank();
  const int team = GRID ? 0 : blockIdx.x / C;
  const int vc = (1 << dC) + c;                 // slab node

  // shared tables: tree (lo, sz) and per-depth offsets of the local q storage
  int* s_lo = reinterpret_cast<int*>(smem_raw);
  int* s_sz = s_lo + a.nnodes;
  int* s_qbase = s_sz + a.nnodes;               // [L+2]
  int* s_leafnode = s_qbase + 32;               // [slab_max]
  size_t hdr = (size_t)(2 * a.nnodes + 32 + a.slab_max) * sizeof(int);
  hdr = (hdr + 15) & ~size_t(15);
  Cx<R>* xs = reinterpret_cast<Cx<R>*>(smem_raw + hdr);        // [2][G][slab_max]
  Cx<R>* qanc = xs + 2 * G_ * a.slab_max;                       // [dC][r_max][G]
  Cx<R>* qloc = qanc + (size_t)(dC > 0 ? dC : 1) * a.r_max * G_;

  for (int v = tid; v < a.nnodes; v += blockDim.x) { s_lo[v] = a.lo[v]; s_sz[v] = a.sz[v]; }
  if (tid == 0) {
    int base = 0;
    for (int d = 0; d <= L; ++d) {
      s_qbase[d] = base;
      if (d > dC) {
        int maxsz = (n + (1 << d) - 1) >> d;
        int qcap = maxsz < a.r_max ? maxsz : a.r_max;
        base += (1 << (d - dC)) * qcap * G_;
      }
    }
  }
  __syncthreads();
  const int lo_c = s_lo[vc], ns = s_sz[vc];
  for (int i = tid; i < ns; i += blockDim.x) {
    int v = vc;
    for (int d = dC; d < L; ++d) v = 2 * v + ((lo_c + i) >= s_lo[2 * v + 1] ? 1 : 0);
    s_leafnode[i] = v;
  }
  __syncthreads();

  const int warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
  const int leaf_first = 1 << L;
  const int nsteps = 2 * n - 1;
  bool alive = true;

  for (int grp = team; grp < a.ngroups && alive; grp += a.nteams) {
    const int g0 = grp * G_;
    const int gcount = (a.nrhs - g0) < G_ ? (a.nrhs - g0) : G_;
    // step-0 input: u_1 = f_1
    for (int it = tid; it < ns * G_; it += blockDim.x) {
      int i = it % ns, g = it / ns;
      Cx<R> v(0, 0);
      if (g < gcount) v = cvt<R>(a.r[(long long)(g0 + g) * a.N + lo_c + i]);
      xs[g * a.slab_max + i] = v;
    }
    __syncthreads();

    for (int s = 0; s < nsteps; ++s) {
      const bool fwd = s < n;
      const int m = fwd ? s : 2 * n - 2 - s;
      const Cx<R>* F = a.fac + (long long)m * a.layer_stride;
      const int* rk = a.rank + (long long)m * a.nnodes;
      Cx<R>* x = xs + (s & 1) * G_ * a.slab_max;
      Cx<R>* xn = xs + ((s + 1) & 1) * G_ * a.slab_max;
      const int par = s & 1;

      // ---- 1. reductions q_v[k][g] = sum_i F_v[i, k] x[g][i] ------------------------
      for (int d = 1; d <= L; ++d) {
        int nodes, rows, qcap, gs;
        if (d <= dC) {
          nodes = 1; rows = ns; qcap = a.r_max;
        } else {
          nodes = 1 << (d - dC);
          rows = (n + (1 << d) - 1) >> d;
          qcap = rows < a.r_max ? rows : a.r_max;
        }
        gs = pow2ceil32(rows);
        const int gpw = 32 / gs;
        const int ngrp = nwarps * gpw;
        const int gid = warp * gpw + lane / gs;
        const int li = lane % gs;
        const int items = nodes * qcap;
        // all lanes of a warp iterate together so that the group shuffles stay converged
        for (int base = 0; base < items; base += ngrp) {
          const int item = base + gid;
          const bool live_item = item < items;
          int v = 0, k = 0, rv = 0, ld = 1, roff = 0, xoff = 0, cnt = 0;
          if (live_item) {
            int j = item / qcap;
            k = item - j * qcap;
            if (d <= dC) {
              v = vc >> (dC - d);
              roff = lo_c - s_lo[v];
              xoff = 0;
              cnt = ns;
            } else {
              v = (vc << (d - dC)) + j;
              roff = 0;
              xoff = s_lo[v] - lo_c;
              cnt = s_sz[v];
            }
            rv = rk[v];
            ld = s_sz[v];
          }
          Cx<R> acc[G];
#pragma unroll
          for (int g = 0; g < G; ++g) acc[g] = Cx<R>(0, 0);
          if (live_item && k < rv) {
            const Cx<R>* col = F + a.off[v] + (long long)k * ld + roff;
            for (int i = li; i < cnt; i += gs) {
              Cx<R> f = col[i];
#pragma unroll
              for (int g = 0; g < G; ++g) cfma(acc[g], f, x[g * a.slab_max + xoff + i]);
            }
          }
#pragma unroll
          for (int g = 0; g < G; ++g)
            for (int o = gs >> 1; o > 0; o >>= 1) acc[g] += shfl_xor(acc[g], o);
          if (live_item && li == 0) {
            int j = item / qcap;
            if (d <= dC) {
              Cx<R>* dst = a.xch + ((((long long)par * a.nteams + team) * dC + (d - 1)) * C + c) * a.r_max * G_;
#pragma unroll
              for (int g = 0; g < G; ++g) st_cg(dst + k * G_ + g, acc[g]);
            } else {
              Cx<R>* dst = qloc + s_qbase[d] + (j * qcap + k) * G_;
#pragma unroll
              for (int g = 0; g < G; ++g) dst[g] = acc[g];
            }
          }
        }
      }

      // ---- 2. team barrier ----------------------------------------------------------
      if (GRID) {
        if (!grid_barrier(a.bar, gridDim.x, a.status, m)) { alive = false; break; }
      } else {
        cg::this_cluster().sync();
      }

      // ---- 3a. sibling sums of the ancestors ----------------------------------------
      for (int it = tid; it < dC * a.r_max * G_; it += blockDim.x) {
        int d = it / (a.r_max * G_) + 1;
        int kg = it - (d - 1) * a.r_max * G_;
        int v = vc >> (dC - d);
        int sib = v ^ 1;
        int span = 1 << (dC - d);
        int c0 = (sib << (dC - d)) - (1 << dC);
        Cx<R> acc(0, 0);
        if (kg / G_ < rk[v]) {
          const Cx<R>* src = a.xch + ((((long long)par * a.nteams + team) * dC + (d - 1)) * C) * a.r_max * G_ + kg;
          for (int cc = 0; cc < span; ++cc) acc += ld_cg(src + (long long)(c0 + cc) * a.r_max * G_);
        }
        qanc[it] = acc;
      }
      __syncthreads();

      // ---- 3b. expansion and the sweep update --------------------------------------
      for (int it = tid; it < ns * G_; it += blockDim.x) {
        const int i = it % ns, g = it / ns;
        const int row = lo_c + i;
        const int lam = s_leafnode[i];
        Cx<R> y(0, 0);
        {
          const Cx<R>* D = F + (long long)(lam - leaf_first) * a.leaf * a.leaf;
          const int lr = row - s_lo[lam], lx = s_lo[lam] - lo_c;
          const int nl = s_sz[lam];
          for (int jj = 0; jj < nl; ++jj) cfma(y, D[lr + jj * a.leaf], x[g * a.slab_max + lx + jj]);
        }
        for (int d = 1; d <= L; ++d) {
          const int v = lam >> (L - d);
          const int rv = rk[v];
          if (rv == 0) continue;
          const int ld = s_sz[v];
          const Cx<R>* col = F + a.off[v] + (row - s_lo[v]);
          const Cx<R>* q;
          if (d <= dC) {
            q = qanc + (d - 1) * a.r_max * G_ + g;
          } else {
            const int maxsz = (n + (1 << d) - 1) >> d;
            const int qcap = maxsz < a.r_max ? maxsz : a.r_max;
            const int jsib = (v ^ 1) - (vc << (d - dC));
            q = qloc + s_qbase[d] + jsib * qcap * G_ + g;
          }
          for (int k = 0; k < rv; ++k) cfma(y, col[(long long)k * ld], q[k * G_]);
        }
        const bool valid = g < gcount;
        const long long p = (long long)(g0 + g) * a.N + (long long)m * n + row;
        if (fwd) {
          if (m < n - 1) {
            Cx<R> f(0, 0);
            if (valid) {
              a.w[p] = y;
              f = cvt<R>(a.r[p + n]);
            }
            Cx<R> cpl = cvt<R>(a.north[(long long)(m + 1) * n + row]);
            xn[g * a.slab_max + i] = f - cpl * y;
          } else {
            if (valid) a.z[p] = cvt<double>(y);
            xn[g * a.slab_max + i] = cvt<R>(a.north[(long long)m * n + row]) * y;
          }
        } else {
          Cx<R> u(0, 0);
          if (valid) {
            u = a.w[p] - y;
            a.z[p] = cvt<double>(u);
          }
          if (m > 0) xn[g * a.slab_max + i] = cvt<R>(a.north[(long long)m * n + row]) * u;
        }
      }
      __syncthreads();
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Host side: team configuration, workspace and launch.

struct SweepConfig {
  bool grid;
  int dC, C, G, nteams;
};

static int ilog2(int x) { int l = 0; while ((1 << (l + 1)) <= x) ++l; return l; }

static SweepConfig choose_config(const hsweep_s* h, int nrhs) {
  SweepConfig cfg{};
  int maxC = h->nleaves;
  int G_opt = h->opt.groups;
  if (h->opt.team > 0) {
    int C = 1 << ilog2(h->opt.team);
    if (C > maxC) C = maxC;
    cfg.C = C;
    cfg.grid = C > 16;
  } else if (h->prec == HSWEEP_FP64 && nrhs <= 2) {
    int C = 64;
    while (C > maxC) C >>= 1;
    cfg.C = C;
    cfg.grid = C > 16;
  } else {
    int C = 16;
    while (C > maxC) C >>= 1;
    cfg.C = C;
    cfg.grid = false;
  }
  cfg.dC = ilog2(cfg.C);
  int team_cap = cfg.grid ? 1 : (h->num_sms / cfg.C > 0 ? h->num_sms / cfg.C : 1);
  int G = 1;
  if (G_opt == 1 || G_opt == 2 || G_opt == 4 || G_opt == 8) {
    G = G_opt;
  } else {
    while (G < 8 && (nrhs + G - 1) / G > team_cap) G <<= 1;
  }
  cfg.G = G;
  int ngroups = (nrhs + G - 1) / G;
  cfg.nteams = cfg.grid ? 1 : (ngroups < team_cap ? ngroups : team_cap);
  return cfg;
}

template <typename R, int G, bool GRID>
static int launch_sweep(hsweep_s* h, const SweepConfig& cfg, SweepArgs<R>& a, size_t smem) {
  auto kern = sweep_kernel<R, G, GRID>;
  HSW_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute at[1];
  lc.blockDim = dim3(kThreads);
  lc.dynamicSmemBytes = smem;
  lc.stream = h->stream;
  if (GRID) {
    lc.gridDim = dim3(cfg.C);
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
  } else {
    if (cfg.C > 8) HSW_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    int nteams = cfg.nteams;
    lc.gridDim = dim3(cfg.C * nteams);
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cfg.C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
  }
  lc.attrs = at;
  lc.numAttrs = 1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (h->prof) {
    for (cudaEvent_t* e : {&e0, &e1}) {
      if (!h->ev_free.empty()) { *e = h->ev_free.back(); h->ev_free.pop_back(); }
      else HSW_CUDA(cudaEventCreate(e));
    }
    HSW_CUDA(cudaEventRecord(e0, h->stream));
  }
  HSW_CUDA(cudaLaunchKernelEx(&lc, kern, a));
  h->nlaunch += 1;
  if (h->prof) {
    HSW_CUDA(cudaEventRecord(e1, h->stream));
    h->ev_sweep.push_back({e0, e1});
  }
  return HSWEEP_OK;
}

template <typename R, bool GRID>
static int dispatch_G(hsweep_s* h, const SweepConfig& cfg, SweepArgs<R>& a, size_t smem) {
  switch (cfg.G) {
    case 1: return launch_sweep<R, 1, GRID>(h, cfg, a, smem);
    case 2: return launch_sweep<R, 2, GRID>(h, cfg, a, smem);
    case 4: return launch_sweep<R, 4, GRID>(h, cfg, a, smem);
    default: return launch_sweep<R, 8, GRID>(h, cfg, a, smem);
  }
}

template <typename R>
static int apply_impl(hsweep_s* h, const c128* r, c128* z, int nrhs, const SweepConfig& cfg) {
  const size_t es = sizeof(Cx<R>);
  long long need_w = (long long)nrhs * h->N;
  if (need_w > h->wcache_cap) {
    int rc = hsw_regrow(h, &h->d_wcache, (size_t)need_w * es);
    if (rc) {
      if (!h->d_wcache) h->wcache_cap = 0;
      return rc;
    }
    h->wcache_cap = need_w;
  }
  long long need_x = 2LL * cfg.nteams * (cfg.dC > 0 ? cfg.dC : 1) * cfg.C * h->r_max * cfg.G;
  if (need_x > h->xch_cap) {
    int rc = hsw_regrow(h, &h->d_xch, (size_t)need_x * es);
    if (rc) {
      if (!h->d_xch) h->xch_cap = 0;
      return rc;
    }
    h->xch_cap = need_x;
  }
  SweepArgs<R> a;
  a.n = h->n; a.L = h->L; a.leaf = h->leaf; a.r_max = h->r_max; a.nnodes = h->nnodes;
  a.dC = cfg.dC; a.C = cfg.C; a.nteams = cfg.nteams; a.nrhs = nrhs;
  a.ngroups = (nrhs + cfg.G - 1) / cfg.G;
  a.slab_max = h->tree.maxsz(cfg.dC);
  a.N = h->N; a.layer_stride = h->layer_stride;
  a.lo = h->d_lo; a.sz = h->d_sz; a.off = h->d_off;
  a.fac = reinterpret_cast<const Cx<R>*>(h->d_fac);
  a.rank = h->d_rank; a.north = h->d_north_m;
  a.r = r; a.z = z;
  a.w = reinterpret_cast<Cx<R>*>(h->d_wcache);
  a.xch = reinterpret_cast<Cx<R>*>(h->d_xch);
  a.status = h->d_status; a.bar = h->d_bar;
  // shared memory: tree tables, x double buffer, ancestor and local q storage
  size_t hdr = (size_t)(2 * h->nnodes + 32 + a.slab_max) * sizeof(int);
  hdr = (hdr + 15) & ~size_t(15);
  long long qloc = 0;
  for (int d = cfg.dC + 1; d <= h->L; ++d) {
    int mx = h->tree.maxsz(d);
    qloc += (long long)(1 << (d - cfg.dC)) * (mx < h->r_max ? mx : h->r_max) * cfg.G;
  }
  size_t smem = hdr + es * (size_t)(2LL * cfg.G * a.slab_max + (long long)(cfg.dC > 0 ? cfg.dC : 1) * h->r_max * cfg.G + qloc);
  if (smem > 227 * 1024) return HSWEEP_ERR_ARG;
  if (cfg.grid) {
    HSW_CUDA(cudaMemsetAsync(h->d_bar, 0, 2 * sizeof(unsigned), h->stream));
    return dispatch_G<R, true>(h, cfg, a, smem);
  }
  return dispatch_G<R, false>(h, cfg, a, smem);
}

int hsw_apply(hsweep_s* h, const c128* r, c128* z, int nrhs) {
  if (nrhs <= 0) return HSWEEP_OK;
  if (h->opt.sweep_kernel == 0 && h->strong_R > 0) {
    bool used = false;
    int rc = hsw_apply_strong(h, r, z, nrhs, &used);
    if (rc != HSWEEP_OK || used) return rc;
  }
  if (h->opt.sweep_kernel != 1) {
    bool used = false;
    int rc = hsw_apply_team(h, r, z, nrhs, &used);
    if (rc != HSWEEP_OK || used) return rc;
  }
  SweepConfig cfg = choose_config(h, nrhs);
  if (h->prec == HSWEEP_FP64) return apply_impl<double>(h, r, z, nrhs, cfg);
  return apply_impl<float>(h, r, z, nrhs, cfg);
}

// ---------------------------------------------------------------------------------------
// The same sweep with caller-provided scratch (the w cache and the team exchange slots
// carved out of one buffer).  Nothing is allocated here.

static long long align_up(long long x, long long a) { return (x + a - 1) / a * a; }

size_t hsw_apply_scratch_bytes(hsweep_s* h, int nrhs) {
  if (nrhs <= 0) return 0;
  if (h->opt.sweep_kernel == 0 && h->strong_R > 0) {
    const size_t fs = hsw_apply_strong_scratch_bytes(h, nrhs);
    if (fs > 0) return fs;
  }
  if (h->opt.sweep_kernel != 1) {
    const size_t fl = hsw_apply_team_scratch_bytes(h, nrhs);
    if (fl > 0) return fl;
  }
  SweepConfig cfg = choose_config(h, nrhs);
  const long long es = h->prec == HSWEEP_FP64 ? (long long)sizeof(c128) : (long long)sizeof(c64);
  const long long w = (long long)nrhs * h->N * es;
  const long long x = 2LL * cfg.nteams * (cfg.dC > 0 ? cfg.dC : 1) * cfg.C * h->r_max * cfg.G * es;
  return (size_t)(align_up(w, 256) + align_up(x, 256));
}

template <typename R>
static int apply_scratch_impl(hsweep_s* h, const c128* r, c128* z, int nrhs, const SweepConfig& cfg,
                              unsigned char* scratch) {
  const size_t es = sizeof(Cx<R>);
  SweepArgs<R> a;
  a.n = h->n; a.L = h->L; a.leaf = h->leaf; a.r_max = h->r_max; a.nnodes = h->nnodes;
  a.dC = cfg.dC; a.C = cfg.C; a.nteams = cfg.nteams; a.nrhs = nrhs;
  a.ngroups = (nrhs + cfg.G - 1) / cfg.G;
  a.slab_max = h->tree.maxsz(cfg.dC);
  a.N = h->N; a.layer_stride = h->layer_stride;
  a.lo = h->d_lo; a.sz = h->d_sz; a.off = h->d_off;
  a.fac = reinterpret_cast<const Cx<R>*>(h->d_fac);
  a.rank = h->d_rank; a.north = h->d_north_m;
  a.r = r; a.z = z;
  a.w = reinterpret_cast<Cx<R>*>(scratch);
  a.xch = reinterpret_cast<Cx<R>*>(scratch + align_up((long long)nrhs * h->N * (long long)es, 256));
  a.status = h->d_status; a.bar = h->d_bar;
  size_t hdr = (size_t)(2 * h->nnodes + 32 + a.slab_max) * sizeof(int);
  hdr = (hdr + 15) & ~size_t(15);
  long long qloc = 0;
  for (int d = cfg.dC + 1; d <= h->L; ++d) {
    int mx = h->tree.maxsz(d);
    qloc += (long long)(1 << (d - cfg.dC)) * (mx < h->r_max ? mx : h->r_max) * cfg.G;
  }
  size_t smem = hdr + es * (size_t)(2LL * cfg.G * a.slab_max + (long long)(cfg.dC > 0 ? cfg.dC : 1) * h->r_max * cfg.G + qloc);
  if (smem > 227 * 1024) return HSWEEP_ERR_ARG;
  const bool prof = h->prof;
  h->prof = false;   // no events are created on this path
  int rc;
  if (cfg.grid) {
    if (cudaMemsetAsync(h->d_bar, 0, 2 * sizeof(unsigned), h->stream) != cudaSuccess) { h->prof = prof; return HSWEEP_ERR_CUDA; }
    rc = dispatch_G<R, true>(h, cfg, a, smem);
  } else {
    rc = dispatch_G<R, false>(h, cfg, a, smem);
  }
  h->prof = prof;
  return rc;
}

int hsw_apply_scratch(hsweep_s* h, const c128* r, c128* z, int nrhs, void* scratch, size_t bytes) {
  if (nrhs <= 0) return HSWEEP_OK;
  if (hsw_apply_scratch_bytes(h, nrhs) > bytes) return HSWEEP_ERR_ARG;
  if (h->opt.sweep_kernel == 0 && h->strong_R > 0) {      // the same kernel hsw_apply would use
    bool used = false;
    int rc = hsw_apply_strong(h, r, z, nrhs, &used, scratch, bytes);
    if (rc != HSWEEP_OK || used) return rc;
  }
  if (h->opt.sweep_kernel != 1) {
    bool used = false;
    int rc = hsw_apply_team(h, r, z, nrhs, &used, scratch, bytes);
    if (rc != HSWEEP_OK || used) return rc;
  }
  SweepConfig cfg = choose_config(h, nrhs);
  if (h->prec == HSWEEP_FP64) return apply_scratch_impl<double>(h, r, z, nrhs, cfg, (unsigned char*)scratch);
  return apply_scratch_impl<float>(h, r, z, nrhs, cfg, (unsigned char*)scratch);
}
