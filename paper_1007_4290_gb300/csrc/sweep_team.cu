// The apply z = M r of Algorithm 2.6 by cooperative teams of CTAs.
//
// A team of C = 2^dC CTAs carries G right-hand sides through the 2n-1 dependent
// hmatvecs of the forward and backward sweeps; CTA c owns the rows of the depth-dC tree
// node vc = 2^dC + c (its slab).  Every CTA of the grid is resident (cooperative launch,
// one CTA per SM), so teams need no thread-block cluster and the whole GPU can be used.
// One step (one layer m, one hmatvec y = T~_m x of Section 2.4 plus the update of
// Algorithm 2.6) runs as:
//   0. the layer's factor record for the slab (leaf-major packed layout, pack.cu) is
//      already in shared memory: warp 0 issued its bulk copy one step ahead (mbarrier),
//      and now issues the next one;
//   1. partial sums q_v = F_v^t x over the slab's rows for the ancestors v at depths
//      1..dC (their rows span several CTAs), stored to L2 with a step tag;
//   2. the reductions of the CTA's own subtree (depths > dC), then
//   3. the gather: the sums over the sibling subtree of every ancestor, read from L2,
//      re-read until every word carries the tag of this step;
//   4. expansion y_i = D x + sum_v F_v[i, :] q_sib(v): eight lanes per row, each over
//      every eighth column, all G right-hand sides in registers;
//   5. the update of Algorithm 2.6 for (row, right-hand side) pairs, one per thread,
//      with coalesced global reads and writes;
//      the row offsets and block tables of the next step's record.
// Three block barriers per step; no team-wide barrier: a CTA waits only for the
// partial sums it reads.  The tag is the lowest bit of every 8-byte word of a partial
// sum, equal to bit 1 of the step index: a slot (one per step parity) holds either
// this step's value or the one from two steps before, because no CTA can run two steps
// ahead of a CTA whose partial sums it reads.  The tag costs one bit of the stored
// mantissa (relative 2^-23 in complex64, 2^-52 in complex128).
// Reductions are warp-items (node, eight columns): lane = (column, one of four row
// subsets), all G right-hand sides per lane, combined by shuffles; warps take items
// from a shared counter.  Vectors in shared memory (x, q, y) are rows of G entries with
// a padded stride, read as 16-byte pairs where G is even.  In complex64 the
// multiply-adds use the paired FP32 instruction fma.rn.f32x2: with a = sum (Re f) x and
// b = sum (Im f) x, f x = (Re a - Im b, Im a + Re b).
#include <cstdlib>
#include <type_traits>
#include "handle.h"
#include "sweep_common.cuh"
#include "tma.cuh"

namespace {

using namespace tma;
using namespace sweepc;

constexpr int kThreads = 512;              // threads of the one-CTA-per-SM variant
constexpr int kThreads2 = 256;             // threads of the two-CTAs-per-SM variant
constexpr int kKS = 8;                      // expansion: lanes (column slices) per row
constexpr int kKW = 8;                      // reduction: column lanes per warp-item
// update pairs (row, right-hand side) per thread: slab rows x G <= kThreads * upt(G)
__host__ __device__ constexpr int upt(int G) { return G >= 8 ? 1 : 2; }
constexpr long long kWaitLimit = 1LL << 22; // bounded waits (about a second)

// ---- tensor cores: mma.sync m16n8k8 with TF32 operands in three parts ---------------
// x = hi + lo: hi is x rounded to the 10 explicit mantissa bits of TF32 (integer add
// and mask, full-rate ALU), lo = x - hi is exact in FP32 and the tensor core reads its
// top TF32 bits; a product is hi*hi + hi*lo + lo*hi in FP32 accumulation (the dropped
// lo*lo term and the truncation of lo are below 2^-21 relative).
__device__ __forceinline__ void split_tf32(float x, unsigned& hi, unsigned& lo) {
  hi = (__float_as_uint(x) + 0x1000u) & 0xffffe000u;
  lo = __float_as_uint(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
// A complex product sum C = sum_k V[k] F[k] over complex k as one real m16n8k8 step:
// A rows 0..7 give the real parts of eight outputs, rows 8..15 the imaginary parts,
// real column 2k + p holds part p of complex index k:
//   A[g][2k] = Re V_g[k], A[g][2k+1] = -Im V_g[k], A[g+8][2k] = Im V_g[k], A[g+8][2k+1] = Re V_g[k]
//   B[2k + p][n] = part p of F_n[k].
// Lane (g = lane / 4, t = lane % 4) holds V_g at complex indices k0 + t/2 (va) and
// k0 + 2 + t/2 (vb); p = t % 2.
struct TcA {
  unsigned h[4], l[4];
  __device__ __forceinline__ void build(Cx<float> va, Cx<float> vb, int p) {
    split_tf32(p ? -va.im : va.re, h[0], l[0]);
    split_tf32(p ? va.re : va.im, h[1], l[1]);
    split_tf32(p ? -vb.im : vb.re, h[2], l[2]);
    split_tf32(p ? vb.re : vb.im, h[3], l[3]);
  }
};
__device__ __forceinline__ void tc_step(float (&c)[4], float (&c2)[4], const TcA& A, float fa, float fb) {
  unsigned bh0, bl0, bh1, bl1;
  split_tf32(fa, bh0, bl0);
  split_tf32(fb, bh1, bl1);
  mma_tf32(c, A.h[0], A.h[1], A.h[2], A.h[3], bh0, bh1);
  mma_tf32(c2, A.l[0], A.l[1], A.l[2], A.l[3], bh0, bh1);
  mma_tf32(c2, A.h[0], A.h[1], A.h[2], A.h[3], bl0, bl1);
}

template <typename R>
struct TeamArgs {
  int n, L, leaf, nnodes, dC, C, nteams, nrhs, ngroups, slab_max, nl, rcap;
  int tc;              // ancestor contractions on tensor cores (complex64, slab <= 64 rows)
  long long N, pack_stride;
  unsigned stage_bytes;
  const int* lo;
  const int* sz;
  const int* rank;
  const long long* recoff;
  const Cx<R>* pack;
  const c128* north;
  const c128* r;
  c128* z;
  Cx<R>* w;
  typename Tagged<R>::W* xch;   // ancestors' tagged partial sums: [2][nteams][C][dC][rcap][G]
  int* status;
  long long wait_limit;         // iterations of the waits for other CTAs' partial sums
                                // (kWaitLimit unless a test shortens it; the waits for this
                                // CTA's own bulk copies always allow kWaitLimit)
  int withhold;                 // test only: this CTA never publishes its partial sums (-1: none)
  int qcapd[16];                // per depth: the largest rank over all layers (capacity of the
                                // shared q slots; the exchanged slots below it are rewritten
                                // every step)
  // shared-memory plan (byte offsets)
  unsigned o_stage[2], o_rowoff[2], o_trk[3], o_ro[3], o_lo, o_sz, o_leafnode, o_dtab, o_wdesc, o_etab[2], o_x[2],
      o_qanc, o_qloc, o_mbar, o_flags;
};

// per-depth table columns in shared memory (16 ints each)
enum { DT_NODES = 0, DT_QCAP = 16, DT_WSTART = 32, DT_QBASE = 48, DT_QANC = 64, DT_SIZE = 80 };

// Reduction of one warp-item: lane (column k, row subset rl) sums rows rb + rl,
// rb + rl + 4, ... < re of column k for all G right-hand sides.
template <typename R, int G, int GS>
__device__ __forceinline__ void reduce_col(const Cx<R>* __restrict__ st, const int* __restrict__ ro_d,
                                           const Cx<R>* __restrict__ x, int rb, int re, int rl, int k,
                                           Cx<R> (&out)[G]) {
  using M = Mac<R>;
  typename M::A acc[G];
#pragma unroll
  for (int g = 0; g < G; ++g) M::zero(acc[g]);
#pragma unroll 4
  for (int i = rb + rl; i < re; i += 32 / kKW) {
    const typename M::F f = M::f(st + ro_d[i] + k);
    typename M::X xv[G];
    load_row<R, G>(x + i * GS, xv);
#pragma unroll
    for (int g = 0; g < G; ++g) M::mac(acc[g], f, xv[g]);
  }
#pragma unroll
  for (int g = 0; g < G; ++g) out[g] = M::get(acc[g]);
}

// Expansion of one row against one vector block: columns k = kbeg, kbeg + KSTEP, ...
// < kend of the row F, vectors V[k * GS + g].
template <typename R, int G, int GS, int KSTEP = kKS>
__device__ __forceinline__ void expand_row(typename Mac<R>::A (&acc)[G], const Cx<R>* __restrict__ F,
                                           const Cx<R>* __restrict__ V, int kbeg, int kend) {
  using M = Mac<R>;
  // not unrolled: a depth's block gives a lane only one to six columns, and the unrolled
  // loop's remainder handling cost more than it saved (measured: 3.9 against 4.2 us of a
  // 64-RHS step's expansion)
#pragma unroll 1
  for (int k = kbeg; k < kend; k += KSTEP) {
    const typename M::F f = M::f(F + k);
    typename M::X v[G];
    load_row<R, G>(V + k * GS, v);
#pragma unroll
    for (int g = 0; g < G; ++g) M::mac(acc[g], f, v[g]);
  }
}

// NT threads per CTA: 512 with one CTA per SM, or 256 with two CTAs per SM (the same
// registers per thread; one CTA's barrier waits and latencies are covered by the other's)
// WIDE: teams of more than 16 CTAs (a sibling subtree spans more than 8 CTAs)
template <typename R, int G, int TC, int NT, bool WIDE = false>
__global__ void __launch_bounds__(NT, kThreads / NT) sweep_team_kernel(TeamArgs<R> a) {
  extern __shared__ __align__(128) unsigned char sm[];
  using M = Mac<R>;
  using T = Tagged<R>;
  constexpr int GS = vstride<R>(G);
  constexpr int kUPT = upt(G);
  constexpr bool kTC = TC > 0 && std::is_same<R, float>::value && NT == kThreads;   // reductions on tensor cores
  constexpr bool kTCE = TC > 1 && std::is_same<R, float>::value && NT == kThreads;  // and the expansion
  constexpr bool tc = kTC;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = a.n, L = a.L, dC = a.dC, nl = a.nl, lf = a.leaf, SM = a.slab_max;
  const int team = blockIdx.x / a.C, c = blockIdx.x % a.C;
  const int vc = (1 << dC) + c;
  const int lam0 = vc << (L - dC);          // first leaf node of the slab
  const int jglob0 = lam0 - (1 << L);       // its leaf index
  const int L1 = L + 1;

  int* s_lo = reinterpret_cast<int*>(sm + a.o_lo);
  int* s_sz = reinterpret_cast<int*>(sm + a.o_sz);
  int* s_leafnode = reinterpret_cast<int*>(sm + a.o_leafnode);
  int* dt = reinterpret_cast<int*>(sm + a.o_dtab);
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(sm + a.o_mbar);
  volatile int* s_fail = reinterpret_cast<volatile int*>(sm + a.o_flags);
  int* s_ctr = reinterpret_cast<int*>(sm + a.o_flags) + 1;     // reduction item counters [2]
  Cx<R>* qanc = reinterpret_cast<Cx<R>*>(sm + a.o_qanc);
  Cx<R>* qloc = reinterpret_cast<Cx<R>*>(sm + a.o_qloc);

  for (int v = tid; v < a.nnodes; v += NT) { s_lo[v] = a.lo[v]; s_sz[v] = a.sz[v]; }
  __syncthreads();
  const int lo_c = s_lo[vc], ns = s_sz[vc];
  if (tid == 0) {
    // reduction warp-items per depth: (node, chunk of kKW columns); ancestors first
    int wsum = 0, qb = 0, qa = 0;
    for (int d = 1; d <= L; ++d) {
      const int rows = d <= dC ? ns : (n + (1 << d) - 1) >> d;
      const int nodes = d <= dC ? 1 : (1 << (d - dC));
      const int qcap = d <= dC ? a.qcapd[d] : min(rows, a.qcapd[d]);
      dt[DT_NODES + d] = nodes;
      dt[DT_QCAP + d] = qcap;
      dt[DT_WSTART + d] = wsum;
      wsum += nodes * ((qcap + kKW - 1) / kKW);
      dt[DT_QBASE + d] = qb;
      dt[DT_QANC + d] = qa;
      if (d > dC) qb += nodes * qcap * GS;
      else qa += qcap * GS;
    }
    dt[DT_WSTART + L + 1] = wsum;
    int* wdesc = reinterpret_cast<int*>(sm + a.o_wdesc);
    int wi = 0;
    for (int d = 1; d <= L; ++d) {
      const int nodes = dt[DT_NODES + d], qcap = dt[DT_QCAP + d];
      const int nkc = (qcap + kKW - 1) / kKW;
      for (int jn = 0; jn < nodes; ++jn)
        for (int kc = 0; kc < nkc; ++kc) wdesc[wi++] = d | (kc << 4) | (jn << 12);
    }
    *s_fail = 0;
    s_ctr[0] = 0;
    s_ctr[1] = 0;
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_mbar_init();
  }
  for (int i = tid; i < ns; i += NT) {
    int v = vc;
    for (int d = dC; d < L; ++d) v = 2 * v + ((lo_c + i) >= s_lo[2 * v + 1] ? 1 : 0);
    s_leafnode[i] = v;
  }
  __syncthreads();

  const int nsteps = 2 * n - 1;
  const int ngroups_team = a.ngroups > team ? (a.ngroups - 1 - team) / a.nteams + 1 : 0;
  const int total_steps = ngroups_team * nsteps;
  auto layer_of = [&](int s) { return s < n ? s : 2 * n - 2 - s; };
  auto inc3 = [](int v) { return v == 2 ? 0 : v + 1; };

  // warp 0: cp.async of the ranks of the slab's nodes and the record offsets of the
  // step at sweep position s into table slot slot3
  auto load_tables = [&](int s, int slot3) {
    const int m = layer_of(s);
    int* trk = reinterpret_cast<int*>(sm + a.o_trk[slot3]);
    long long* sro = reinterpret_cast<long long*>(sm + a.o_ro[slot3]);
    const int* rk = a.rank + (long long)m * a.nnodes;
    const long long* ro = a.recoff + (long long)m * ((long long)(1 << L) + 1);
    const int nloc = 2 * nl - 2;
    for (int q = lane; q < dC + nloc + nl + 1; q += 32) {
      if (q < dC) {
        cp_async4(trk + q, rk + (vc >> (dC - 1 - q)));
      } else if (q < dC + nloc) {
        const int li = q - dC;
        int dd = 1;
        while ((1 << (dd + 1)) - 2 <= li) ++dd;
        cp_async4(trk + q, rk + (vc << dd) + (li - ((1 << dd) - 2)));
      } else {
        const int j = q - dC - nloc;
        cp_async8(sro + j, ro + jglob0 + j);
      }
    }
  };
  // threads w0, w0 + wn, ...: from the ranks and record offsets in table slot slot3, the
  // offset of every row of every block of that step's record (rowoff buffer rb), and per
  // (slab leaf, depth) the rank and the shared-memory vector block the expansion multiplies
  // it with (etab buffer eb)
  auto build_tables = [&](int slot3, int eb, int rb, int w0, int wn) {
    const int* trk = reinterpret_cast<const int*>(sm + a.o_trk[slot3]);
    const long long* sro = reinterpret_cast<const long long*>(sm + a.o_ro[slot3]);
    int* rowoff = reinterpret_cast<int*>(sm + a.o_rowoff[rb]);
    int* erk = reinterpret_cast<int*>(sm + a.o_etab[eb]);
    int* evo = erk + nl * L1;
    auto rank_at = [&](int lam, int d) {
      return d <= dC ? trk[d - 1] : trk[dC + (1 << (d - dC)) - 2 + ((lam >> (L - d)) - (vc << (d - dC)))];
    };
    for (int e = w0; e < ns * L1; e += wn) {
      const int i = e % ns, d = e / ns;
      const int lam = s_leafnode[i];
      const int j = lam - lam0;
      const int sl = s_sz[lam], ai = lo_c + i - s_lo[lam];
      int o = (int)(sro[j] - sro[0]);
      if (d == 0) {
        o += ai * lf;
      } else {
        o += lf * lf;
        for (int dd = 1; dd < d; ++dd) o += sl * row_stride(rank_at(lam, dd));
        o += ai * row_stride(rank_at(lam, d));
      }
      rowoff[d * SM + i] = o;
    }
    for (int e = w0; e < nl * L1; e += wn) {
      const int j = e / L1, d = e % L1;
      const int lam = lam0 + j;
      int r, vo = 0;
      if (d == 0) {
        r = s_sz[lam];
      } else {
        r = rank_at(lam, d);
        if (d <= dC) {
          vo = (int)a.o_qanc + (int)sizeof(Cx<R>) * dt[DT_QANC + d];
        } else {
          const int jn = (lam >> (L - d)) - (vc << (d - dC));
          vo = (int)a.o_qloc + (int)sizeof(Cx<R>) * (dt[DT_QBASE + d] + ((jn ^ 1) * dt[DT_QCAP + d]) * GS);
        }
      }
      erk[e] = r;
      evo[e] = vo;
    }
  };
  // warp 0, lane 0: the bulk copy of the record of sweep position s (tables in slot3)
  // into stage `slot`
  auto produce = [&](int s, int slot3, int slot) {
    if (lane != 0) return;
    const int m = layer_of(s);
    const long long* sro = reinterpret_cast<const long long*>(sm + a.o_ro[slot3]);
    const unsigned bytes = (unsigned)((sro[nl] - sro[0]) * (long long)sizeof(Cx<R>));
    unsigned long long* mb = &mbar[slot];
    if (bytes > a.stage_bytes || bytes == 0) {
      if (bytes > a.stage_bytes) report_error(a.status, HSWEEP_ERR_ARG, m);
      mbar_arrive(mb);      // complete the phase without data
    } else {
      fence_proxy_async();
      mbar_expect_tx(mb, bytes);
      bulk_g2s(sm + a.o_stage[slot], a.pack + (long long)m * a.pack_stride + sro[0], bytes, mb);
    }
  };

  if (warp == 0 && total_steps > 0) {
    load_tables(0, 0);
    if (total_steps > 1) load_tables(1, 1);
    cp_async_commit();
    cp_async_wait0();
    __syncwarp();
    produce(0, 0, 0);
  }
  __syncthreads();
  if (total_steps > 0) build_tables(0, 0, 0, tid, NT);
  __syncthreads();

  int issued = total_steps > 0 ? 1 : 0;   // bulk copies issued (steps 0 .. issued-1)
  int t = 0, s = 0, grp = team, slot3 = 0;   // slot3 = t % 3
  for (; t < total_steps; ++t) {
    const int g0 = grp * G;
    const int gcount = (a.nrhs - g0) < G ? (a.nrhs - g0) : G;
    const bool fwd = s < n;
    const int m = fwd ? s : 2 * n - 2 - s;
    const int slot = t & 1;
    const unsigned tag = (unsigned)(t >> 1) & 1u;
    Cx<R>* x = reinterpret_cast<Cx<R>*>(sm + a.o_x[s & 1]);
    Cx<R>* xn = reinterpret_cast<Cx<R>*>(sm + a.o_x[(s + 1) & 1]);
    // the expansion's result y is held in the next step's x buffer: the update reads
    // y[i][g] and then writes x_next[i][g] in the same thread
    Cx<R>* ybuf = xn;
    if (s == 0) {     // a new group: x = r restricted to layer 0 and the slab's rows
      for (int it = tid; it < ns * G; it += NT) {
        const int i = it / G, g = it % G;
        Cx<R> v(0, 0);
        if (g < gcount) v = cvt<R>(a.r[(long long)(g0 + g) * a.N + lo_c + i]);
        x[i * GS + g] = v;
      }
      __syncthreads();
    }
    {   // the stage of step t
      long long spins = 0;
      const unsigned parity = (unsigned)((t >> 1) & 1);
      while (!mbar_try_wait(&mbar[slot], parity)) {
        if (++spins > kWaitLimit) {
          report_error(a.status, HSWEEP_ERR_TIMEOUT, m);
          *s_fail = 1;
          break;
        }
      }
    }
    const Cx<R>* st = reinterpret_cast<const Cx<R>*>(sm + a.o_stage[slot]);
    const int* rowoff = reinterpret_cast<const int*>(sm + a.o_rowoff[t & 1]);
    const int* trk = reinterpret_cast<const int*>(sm + a.o_trk[slot3]);
    const int* wdesc = reinterpret_cast<const int*>(sm + a.o_wdesc);
    const int* erk = reinterpret_cast<const int*>(sm + a.o_etab[slot]);
    const int* evo = erk + nl * L1;
    typename T::W* xpart = a.xch + ((long long)slot * a.nteams + team) * a.C * dC * a.rcap * G;

    // reduction warp-items [wb, we), taken from the shared counter s_ctr[which]
    auto reduce_items = [&](int wb, int we, int which) {
      const int kl = lane % kKW, rl = lane / kKW;
      for (;;) {
        int wi = 0;
        if (lane == 0) wi = atomicAdd(&s_ctr[which], 1);
        wi = __shfl_sync(0xffffffffu, wi, 0) + wb;
        if (wi >= we) break;
        const int desc = wdesc[wi];
        const int d = desc & 15, kc = (desc >> 4) & 255, jn = (desc >> 12) & 4095;
        const int nodes = dt[DT_NODES + d], qcap = dt[DT_QCAP + d];
        const int k = kc * kKW + kl;
        int r, rb, re;
        if (d <= dC) {
          r = trk[d - 1];
          rb = 0;
          re = ns;
        } else {
          const int v = (vc << (d - dC)) + jn;
          r = trk[dC + nodes - 2 + jn];
          rb = s_lo[v] - lo_c;
          re = rb + s_sz[v];
        }
        // every exchanged slot below qcap is rewritten every step (zero past the rank),
        // so a slot never holds a value older than two steps
        Cx<R> out[G];
        if (kc * kKW < r) {
          reduce_col<R, G, GS>(st, rowoff + d * SM, x, rb, re, rl, min(k, r - 1), out);
#pragma unroll
          for (int g = 0; g < G; ++g)
#pragma unroll
            for (int o = kKW; o < 32; o <<= 1) out[g] += shfl_xor(out[g], o);
        } else {
          if (d > dC) continue;           // a subtree item wholly past the rank
#pragma unroll
          for (int g = 0; g < G; ++g) out[g] = Cx<R>(0, 0);
        }
        if (rl == 0 && k < qcap && (k < r || d <= dC)) {
          if (d <= dC) {
            typename T::W* dst = xpart + ((long long)c * dC + (d - 1)) * a.rcap * G + k * G;
            if ((int)blockIdx.x != a.withhold)
#pragma unroll
              for (int g = 0; g < G; ++g) T::store(dst + g, T::pack(k < r ? out[g] : Cx<R>(0, 0), tag));
          } else {
            Cx<R>* dst = qloc + dt[DT_QBASE + d] + (jn * qcap + k) * GS;
#pragma unroll
            for (int g = 0; g < G; ++g) dst[g] = out[g];
          }
        }
      }
    };

    // ---- 0.-3. warp 0: next bulk copy and tables; all warps: ancestor partial sums,
    //            subtree reductions, then the gather of the sibling subtrees' sums ----
    const bool ok1 = *s_fail == 0;
    if (warp == 0 && ok1 && t + 1 < total_steps) {
      const int s1 = s + 1 == nsteps ? 0 : s + 1;
      produce(s1, inc3(slot3), slot ^ 1);
      if (t + 2 < total_steps) {
        load_tables(s1 + 1 == nsteps ? 0 : s1 + 1, inc3(inc3(slot3)));
        cp_async_commit();
      }
      issued = t + 2;
      // the global inputs of step t + 1's update (the coupling row, and per right-hand side
      // the next layer's rows of r or the cached rows of w) into L2 a step ahead: they are
      // read once per launch, from HBM, at the end of a step
      {
        const bool fwd1 = s1 < n;
        const int m1 = fwd1 ? s1 : 2 * n - 2 - s1;
        const int g01 = (s1 == 0 ? grp + a.nteams : grp) * G;
        const int gc1 = max(0, min(G, a.nrhs - g01));
        const int mn1 = (fwd1 && m1 < n - 1) ? m1 + 1 : m1;
        const bool rin = fwd1 && m1 < n - 1;
        const int lines_c = (ns * (int)sizeof(c128) + 127) >> 7;
        const int lines_v = rin ? lines_c : (!fwd1 ? (ns * (int)sizeof(Cx<R>) + 127) >> 7 : 0);
        const int tot = lines_c + gc1 * lines_v;
        for (int q = lane; q < tot; q += 32) {
          if (q < lines_c) {
            prefetch_l2(reinterpret_cast<const unsigned char*>(a.north + (long long)mn1 * n + lo_c) + 128 * q);
          } else {
            const int g = (q - lines_c) / lines_v, l = (q - lines_c) % lines_v;
            const long long row = (long long)(g01 + g) * a.N;
            if (rin) prefetch_l2(reinterpret_cast<const unsigned char*>(a.r + row + (long long)(m1 + 1) * n + lo_c) + 128 * l);
            else prefetch_l2(reinterpret_cast<const unsigned char*>(a.w + row + (long long)m1 * n + lo_c) + 128 * l);
          }
        }
      }
    }
    // ancestors' partial sums on tensor cores: warp-items (depth d, 16 columns), the
    // columns as two n-tiles, the slab's rows as the k dimension
    auto reduce_anc_tc = [&]() {
      if constexpr (kTC) {
        const int g = lane >> 2, tq = lane & 3, pp = tq & 1;
        const int nct = (a.rcap + 15) / 16;
        for (;;) {
          int wi = 0;
          if (lane == 0) wi = atomicAdd(&s_ctr[0], 1);
          wi = __shfl_sync(0xffffffffu, wi, 0);
          if (wi >= dC * nct) break;
          const int d = wi / nct + 1, k0 = (wi % nct) * 16;
          const int r = trk[d - 1];
          float cc[2][4] = {}, c2[2][4] = {};
          if (k0 < r) {
            const int* ro_d = rowoff + d * SM;
            for (int i0 = 0; i0 < ns; i0 += 4) {
              const int ia = i0 + (tq >> 1), ib = ia + 2;
              const Cx<float> va = (ia < ns && g < G) ? x[ia * GS + g] : Cx<float>(0.f, 0.f);
              const Cx<float> vb = (ib < ns && g < G) ? x[ib * GS + g] : Cx<float>(0.f, 0.f);
              TcA A;
              A.build(va, vb, pp);
              const float* Fa = reinterpret_cast<const float*>(st + (ia < ns ? ro_d[ia] : 0)) + pp;
              const float* Fb = reinterpret_cast<const float*>(st + (ib < ns ? ro_d[ib] : 0)) + pp;
#pragma unroll
              for (int nt = 0; nt < 2; ++nt) {
                const int kk = k0 + 8 * nt + g;
                const float fa = (ia < ns && kk < r) ? Fa[2 * kk] : 0.f;
                const float fb = (ib < ns && kk < r) ? Fb[2 * kk] : 0.f;
                tc_step(cc[nt], c2[nt], A, fa, fb);
              }
            }
          }
          // every slot below rcap is rewritten (zero past the rank)
          if (g < G) {
            typename T::W* dst = xpart + ((long long)c * dC + (d - 1)) * a.rcap * G + g;
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
              const int kk = k0 + 8 * nt + 2 * tq;
              if (kk < a.rcap)
                T::store(dst + kk * G, T::pack(Cx<float>(cc[nt][0] + c2[nt][0], cc[nt][2] + c2[nt][2]), tag));
              if (kk + 1 < a.rcap)
                T::store(dst + (kk + 1) * G, T::pack(Cx<float>(cc[nt][1] + c2[nt][1], cc[nt][3] + c2[nt][3]), tag));
            }
          }
        }
      }
    };

    if (ok1) {
      if (tc) reduce_anc_tc();
      else reduce_items(0, dt[DT_WSTART + dC + 1], 0);
      reduce_items(dt[DT_WSTART + dC + 1], dt[DT_WSTART + L + 1], 1);
      // the row offsets and block tables of step t + 1 (buffers step t does not read),
      // while the other CTAs' partial sums are on their way
      if (t + 1 < total_steps) build_tables(inc3(slot3), slot ^ 1, (t + 1) & 1, tid, NT);
      constexpr int GJ = sizeof(R) == 4 ? 3 : 1;
      const int rg = a.rcap * G;
      const int tot = dC * rg;
      const long long cstride = (long long)dC * rg;
      const typename T::W* xb = a.xch + ((long long)slot * a.nteams + team) * a.C * cstride;
      for (int base = tid; base < tot; base += GJ * NT) {
        typename T::W vals[GJ][8];
        const typename T::W* src[GJ];
        int span[GJ];
        bool use[GJ];
#pragma unroll
        for (int j = 0; j < GJ; ++j) {
          const int it = base + j * NT;
          const int d = it < tot ? it / rg + 1 : 1;
          const int kg = it - (d - 1) * rg;
          span[j] = 1 << (dC - d);
          const int c0 = (((vc >> (dC - d)) ^ 1) << (dC - d)) - (1 << dC);
          use[j] = it < tot && kg / G < trk[d - 1];
          src[j] = xb + (long long)(d - 1) * rg + kg + (long long)c0 * cstride;
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (use[j] && u < span[j]) vals[j][u] = T::load(src[j] + u * cstride);
        }
        // re-read every word not yet written for this step, all of them together per round
        {
          long long spins = 0;
          for (;;) {
            bool pending = false;
#pragma unroll
            for (int j = 0; j < GJ; ++j)
#pragma unroll
              for (int u = 0; u < 8; ++u)
                if (use[j] && u < span[j] && !T::ok(vals[j][u], tag)) {
                  vals[j][u] = T::load(src[j] + u * cstride);
                  pending = true;
                }
            if (!pending) break;
            if (++spins > a.wait_limit || *(volatile int*)a.status != 0) {
              report_error(a.status, HSWEEP_ERR_TIMEOUT, m);
              *s_fail = 1;
              break;
            }
          }
        }
#pragma unroll
        for (int j = 0; j < GJ; ++j) {
          const int it = base + j * NT;
          if (it >= tot) continue;
          Cx<R> acc(0, 0);
          if (use[j]) {
#pragma unroll
            for (int u = 0; u < 8; ++u)
              if (u < span[j]) acc += T::value(vals[j][u]);
            if constexpr (WIDE) {
              // teams of more than 16 CTAs: the remaining sources eight at a time, the eight
              // loads in flight together
              for (int u0 = 8; u0 < span[j]; u0 += 8) {
                typename T::W v8[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                  if (u0 + u < span[j]) v8[u] = T::load(src[j] + (u0 + u) * cstride);
                long long spins = 0;
                for (;;) {
                  bool pending = false;
#pragma unroll
                  for (int u = 0; u < 8; ++u)
                    if (u0 + u < span[j] && !T::ok(v8[u], tag)) {
                      v8[u] = T::load(src[j] + (u0 + u) * cstride);
                      pending = true;
                    }
                  if (!pending) break;
                  if (++spins > a.wait_limit || *(volatile int*)a.status != 0) {
                    report_error(a.status, HSWEEP_ERR_TIMEOUT, m);
                    *s_fail = 1;
                    break;
                  }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u)
                  if (u0 + u < span[j]) acc += T::value(v8[u]);
              }
            }
          }
          const int d = it / rg + 1;
          const int kg = it - (d - 1) * rg;
          if (kg / G < dt[DT_QCAP + d]) qanc[dt[DT_QANC + d] + (kg / G) * GS + kg % G] = acc;
        }
      }
    }
    __syncthreads();
    if (*s_fail != 0) break;

    // ---- 4. expansion ----------------------------------------------------------------
    if (kTCE) {
      if constexpr (kTCE) {
        // warps 0..3: the ancestors' terms on tensor cores, rows 16 w .. 16 w + 15 as two
        // n-tiles, the columns of depths 1..dC as the k dimension; warps 4..11: the leaf
        // block and the subtree depths on CUDA cores, four lanes per row
        constexpr int KSL = 4;
        Cx<R> yl[G];
        int iloc = -1;
        if (warp < 4) {
          const int g = lane >> 2, tq = lane & 3, pp = tq & 1;
          float cc[2][4] = {}, c2[2][4] = {};
          const int rA = 16 * warp + g, rB = rA + 8;
          for (int d = 1; d <= dC; ++d) {
            const int r = trk[d - 1];
            const Cx<float>* q = qanc + dt[DT_QANC + d];
            const float* Fa = reinterpret_cast<const float*>(st + (rA < ns ? rowoff[d * SM + rA] : 0)) + pp;
            const float* Fb = reinterpret_cast<const float*>(st + (rB < ns ? rowoff[d * SM + rB] : 0)) + pp;
            for (int k0 = 0; k0 < r; k0 += 4) {
              const int ka = k0 + (tq >> 1), kb = ka + 2;
              const Cx<float> va = (ka < r && g < G) ? q[ka * GS + g] : Cx<float>(0.f, 0.f);
              const Cx<float> vb = (kb < r && g < G) ? q[kb * GS + g] : Cx<float>(0.f, 0.f);
              TcA A;
              A.build(va, vb, pp);
              tc_step(cc[0], c2[0], A, (rA < ns && ka < r) ? Fa[2 * ka] : 0.f, (rA < ns && kb < r) ? Fa[2 * kb] : 0.f);
              tc_step(cc[1], c2[1], A, (rB < ns && ka < r) ? Fb[2 * ka] : 0.f, (rB < ns && kb < r) ? Fb[2 * kb] : 0.f);
            }
          }
          if (g < G) {
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
              const int row = 16 * warp + 8 * nt + 2 * tq;
              if (row < ns) ybuf[row * GS + g] = Cx<R>(cc[nt][0] + c2[nt][0], cc[nt][2] + c2[nt][2]);
              if (row + 1 < ns) ybuf[(row + 1) * GS + g] = Cx<R>(cc[nt][1] + c2[nt][1], cc[nt][3] + c2[nt][3]);
            }
          }
        } else if (warp < 4 + (64 * KSL) / 32) {
          const int lt = tid - 128;
          const int ks = lt % KSL;
          const int i = lt / KSL;
          typename M::A acc[G];
#pragma unroll
          for (int g = 0; g < G; ++g) M::zero(acc[g]);
          if (i < ns) {
            const int lam = s_leafnode[i];
            const int j = lam - lam0;
            const int ib = s_lo[lam] - lo_c;
            const int* eb = erk + j * L1;
            const int* ev = evo + j * L1;
            expand_row<R, G, GS, KSL>(acc, st + rowoff[i], x + ib * GS, ks, eb[0]);
            for (int d = dC + 1; d <= L; ++d)
              expand_row<R, G, GS, KSL>(acc, st + rowoff[d * SM + i], reinterpret_cast<const Cx<R>*>(sm + ev[d]), ks,
                                        eb[d]);
          }
#pragma unroll
          for (int g = 0; g < G; ++g) {
            yl[g] = M::get(acc[g]);
#pragma unroll
            for (int o = 1; o < KSL; o <<= 1) yl[g] += shfl_xor(yl[g], o);
          }
          if (ks == 0 && i < ns) iloc = i;
        }
        __syncthreads();
        if (iloc >= 0) {
#pragma unroll
          for (int g = 0; g < G; ++g) ybuf[iloc * GS + g] += yl[g];
        }
      }
    } else {
      // lane = (row i, column slice ks), all depths on CUDA cores
      const int nitems = ns * kKS;
      for (int item = tid; item < ((nitems + 31) & ~31); item += NT) {
        const bool live = item < nitems;
        const int ks = item % kKS;
        const int i = live ? item / kKS : 0;
        const int lam = s_leafnode[i];
        const int j = lam - lam0;
        const int ib = s_lo[lam] - lo_c;               // first slab row of the leaf
        typename M::A acc[G];
#pragma unroll
        for (int g = 0; g < G; ++g) M::zero(acc[g]);
        if (live) {
          const int* eb = erk + j * L1;
          const int* ev = evo + j * L1;
          expand_row<R, G, GS>(acc, st + rowoff[i], x + ib * GS, ks, eb[0]);
          for (int d = 1; d <= L; ++d)
            expand_row<R, G, GS>(acc, st + rowoff[d * SM + i], reinterpret_cast<const Cx<R>*>(sm + ev[d]), ks, eb[d]);
        }
        Cx<R> y[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          y[g] = M::get(acc[g]);
#pragma unroll
          for (int o = 1; o < kKS; o <<= 1) y[g] += shfl_xor(y[g], o);
        }
        if (live && ks == 0) {
#pragma unroll
          for (int g = 0; g < G; ++g) ybuf[i * GS + g] = y[g];
        }
      }
    }
    // the update's global inputs for this thread's (row, rhs) pairs, issued before the
    // barrier so that their latency overlaps the wait for the slowest warp (issued at the
    // start of the step they cost more issue stalls than they saved)
    c128 pcpl[kUPT], pin[kUPT];
    Cx<R> pw[kUPT];
#pragma unroll
    for (int u = 0; u < kUPT; ++u) {
      const int p = tid + u * NT;
      pcpl[u] = c128(0.0, 0.0);
      pin[u] = c128(0.0, 0.0);
      pw[u] = Cx<R>(0, 0);
      if (p < ns * G) {
        const int i = p % ns, g = p / ns;
        const int mn = (fwd && m < n - 1) ? m + 1 : m;
        pcpl[u] = a.north[(long long)mn * n + lo_c + i];
        if (g < gcount) {
          if (fwd && m < n - 1) pin[u] = a.r[(long long)(g0 + g) * a.N + (long long)(m + 1) * n + lo_c + i];
          else if (!fwd) pw[u] = a.w[(long long)(g0 + g) * a.N + (long long)m * n + lo_c + i];
        }
      }
    }
    __syncthreads();

    // ---- 5. the update of Algorithm 2.6 for this thread's (row, rhs) pairs; the next
    //         step's row offsets ---------------------------------------------------------
#pragma unroll
    for (int u = 0; u < kUPT; ++u) {
      const int p = tid + u * NT;
      if (p < ns * G) {
        const int i = p % ns, g = p / ns;
        const bool valid = g < gcount;
        const c128 fin = pin[u];
        const Cx<R> win = pw[u];
        const Cx<R> y = ybuf[i * GS + g];
        const Cx<R> cpl = cvt<R>(pcpl[u]);
        const long long pos = (long long)(g0 + g) * a.N + (long long)m * n + lo_c + i;
        if (fwd) {
          if (m < n - 1) {
            if (valid) a.w[pos] = y;
            xn[i * GS + g] = cvt<R>(fin) - cpl * y;
          } else {
            if (valid) a.z[pos] = cvt<double>(y);
            xn[i * GS + g] = cpl * y;
          }
        } else {
          const Cx<R> uu = valid ? win - y : Cx<R>(0, 0);
          if (valid) a.z[pos] = cvt<double>(uu);
          if (m > 0) xn[i * GS + g] = cpl * uu;
        }
      }
    }
    if (tid == 0) { s_ctr[0] = 0; s_ctr[1] = 0; }
    // the tables of step t + 2 (cp.async, issued at the start of this step) land before the
    // barrier, so that step t + 1 can build its successor's row offsets from them
    if (warp == 0) cp_async_wait0();
    __syncthreads();
    if (++s == nsteps) { s = 0; grp += a.nteams; }
    slot3 = inc3(slot3);
  }
  // a CTA that stopped early still owns the bulk copies it issued: wait for them
  if (tid == 0) {
    for (int q = t + 1; q < issued; ++q) {
      long long spins = 0;
      const unsigned parity = (unsigned)((q >> 1) & 1);
      while (!mbar_try_wait(&mbar[q & 1], parity) && ++spins <= kWaitLimit) {
      }
    }
  }
  __syncthreads();
}

}  // namespace

namespace {

struct TeamConfig {
  bool ok;
  int dC, C, G, nteams;
  size_t smem;
  int nt;              // threads per CTA (kThreads or kThreads2)
};

static int ilog2t(int x) { int l = 0; while ((1 << (l + 1)) <= x) ++l; return l; }

// shared-memory plan for (dC, G); returns total bytes (0 if the layout is not supported)
template <typename R>
static size_t plan_team(const hsweep_s* h, int dC, int G, TeamArgs<R>& a, int nt = kThreads) {
  const size_t es = sizeof(Cx<R>);
  const int L = h->L;
  const int nl = 1 << (L - dC);
  const int slab_max = h->tree.maxsz(dC);
  const int rcap = std::max(1, h->rank_max);
  const int GS = vstride<R>(G);
  if (L > 14 || (long long)slab_max * G > (long long)upt(G) * nt || h->leaf > 8) return 0;
  auto al = [](size_t x, size_t b) { return (x + b - 1) / b * b; };
  size_t o = 0;
  const size_t stage = al((size_t)h->slab_bytes_max[dC], 128);
  for (int b = 0; b < 2; ++b) { a.o_stage[b] = (unsigned)o; o += stage; }
  for (int b = 0; b < 2; ++b) { a.o_rowoff[b] = (unsigned)o; o += al((size_t)(L + 1) * slab_max * sizeof(int), 16); }
  for (int b = 0; b < 3; ++b) { a.o_trk[b] = (unsigned)o; o += al((size_t)(dC + 2 * nl) * sizeof(int), 16); }
  for (int b = 0; b < 3; ++b) { a.o_ro[b] = (unsigned)o; o += al((size_t)(nl + 1) * sizeof(long long), 16); }
  a.o_lo = (unsigned)o; o += al(h->nnodes * sizeof(int), 16);
  a.o_sz = (unsigned)o; o += al(h->nnodes * sizeof(int), 16);
  a.o_leafnode = (unsigned)o; o += al(slab_max * sizeof(int), 16);
  a.o_dtab = (unsigned)o; o += al(DT_SIZE * sizeof(int), 16);
  long long wtot = 0, qloc = 0, qanc = 0;
  for (int d = 0; d < 16; ++d)
    a.qcapd[d] = d <= L && d < (int)h->rank_max_depth.size() ? std::min(rcap, h->rank_max_depth[d]) : 0;
  for (int d = 1; d <= L; ++d) {
    const int rows = d <= dC ? slab_max : h->tree.maxsz(d);
    const int nodes = d <= dC ? 1 : (1 << (d - dC));
    const int qcap = d <= dC ? a.qcapd[d] : std::min(rows, a.qcapd[d]);
    wtot += (long long)nodes * ((qcap + kKW - 1) / kKW);
    if (d > dC) qloc += (long long)nodes * qcap * GS;
    else qanc += (long long)qcap * GS;
  }
  a.o_wdesc = (unsigned)o; o += al((size_t)wtot * sizeof(int), 16);
  for (int b = 0; b < 2; ++b) { a.o_etab[b] = (unsigned)o; o += al((size_t)2 * nl * (L + 1) * sizeof(int), 16); }
  for (int b = 0; b < 2; ++b) { a.o_x[b] = (unsigned)o; o += al((size_t)slab_max * GS * es, 16); }
  a.o_qanc = (unsigned)o; o += al((size_t)std::max(1LL, qanc) * es, 16);
  a.o_qloc = (unsigned)o; o += al((size_t)std::max(1LL, qloc) * es, 16);
  a.o_mbar = (unsigned)o; o += 16;
  a.o_flags = (unsigned)o; o += 16;
  a.stage_bytes = (unsigned)stage;
  a.nl = nl;
  a.slab_max = slab_max;
  a.rcap = rcap;
  return o;
}

template <typename R, int G, int NT>
static int resident_ctas(const hsweep_s* h, size_t smem) {
  auto kern = sweep_team_kernel<R, G, 0, NT>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * h->num_sms;
}

template <typename R, int NT>
static int resident_for_nt(const hsweep_s* h, int G, size_t smem) {
  switch (G) {
    case 1: return resident_ctas<R, 1, NT>(h, smem);
    case 2: return resident_ctas<R, 2, NT>(h, smem);
    case 4: return resident_ctas<R, 4, NT>(h, smem);
    case 5: return resident_ctas<R, 5, NT>(h, smem);
    default: return resident_ctas<R, 8, NT>(h, smem);
  }
}

template <typename R>
static int resident_for(const hsweep_s* h, int G, size_t smem, int nt) {
  return nt == kThreads2 ? resident_for_nt<R, kThreads2>(h, G, smem) : resident_for_nt<R, kThreads>(h, G, smem);
}

// Team size C, right-hand sides per team G and threads per CTA: the fewest rounds of 2n-1
// dependent steps, a step costing a fixed latency (exchange through L2, barriers, growing
// slowly with the team's depth) plus work that grows with the slab's rows times G per thread.
// Two CTAs of 256 threads on one SM cover each other's barrier waits and latencies: their
// work term is weighted by kShare2.  Coefficients from the measured apply at n = 1023: one
// RHS 12.6 ms with teams of 32 CTAs against 13.4 ms with 16 (complex128: 31.4 ms with 64 CTAs
// against 35.7 ms with 32); 16 RHS 15.0 ms with 16 CTAs and G = 2 against 16.7 ms with 32 CTAs
// and G = 4; 64 RHS 25.8 ms with 16 CTAs and G = 8.
constexpr double kShare2 = 1.5;

template <typename R>
static TeamConfig choose_team_uncached(const hsweep_s* h, int nrhs) {
  TeamConfig best{};
  best.ok = false;
  double best_cost = 1e300;
  const size_t cap = 227 * 1024;
  const int C_pref = h->opt.team, G_pref = h->opt.groups, T_pref = h->opt.team_threads;
  for (int C = 1; C <= h->nleaves && C <= 2 * h->num_sms; C *= 2) {
    if (C_pref > 0 && C != (1 << ilog2t(C_pref))) continue;
    const int dC = ilog2t(C);
    for (int nt : {kThreads, kThreads2}) {
      if (T_pref > 0 && nt != T_pref) continue;
      for (int G : {8, 5, 4, 2, 1}) {
        if (G_pref > 0 && G != G_pref) continue;
        TeamArgs<R> a;
        const size_t smem = plan_team<R>(h, dC, G, a, nt);
        if (smem == 0 || smem > cap) continue;
        const int resident = resident_for<R>(h, G, smem, nt);
        const int teams_cap = std::min(resident, 1024) / C;
        if (teams_cap < 1) continue;
        // the two-CTA variant only where two CTAs per SM are resident
        if (nt == kThreads2 && resident < 2 * h->num_sms) continue;
        const int ngroups = (nrhs + G - 1) / G;
        const int teams = std::min(ngroups, teams_cap);
        const int rounds = (ngroups + teams - 1) / teams;
        const double es = (double)sizeof(Cx<R>) / 8.0;
        const double work = 0.012 * es * a.slab_max * G * ((double)kThreads / nt) * (nt == kThreads2 ? kShare2 : 1.0);
        const double step = 2.5 + work + 0.05 * dC + 0.01 * C;
        const double cost = rounds * step;
        if (cost < best_cost - 1e-9) {
          best_cost = cost;
          best = TeamConfig{true, dC, C, G, teams, smem, nt};
        }
      }
    }
  }
  return best;
}

// the plan for nrhs, from the handle's cache when this nrhs was planned before (the
// occupancy queries behind a plan cost more than a short apply)
template <typename R>
static TeamConfig choose_team(hsweep_s* h, int nrhs) {
  for (const auto& e : h->team_plans)
    if (e[0] == nrhs) return TeamConfig{e[1] != 0, (int)e[2], (int)e[3], (int)e[4], (int)e[5], (size_t)e[6], (int)e[7]};
  const TeamConfig c = choose_team_uncached<R>(h, nrhs);
  if (h->team_plans.size() >= 64) h->team_plans.erase(h->team_plans.begin());
  h->team_plans.push_back({nrhs, c.ok ? 1 : 0, c.dC, c.C, c.G, c.nteams, (long long)c.smem, c.nt});
  return c;
}

template <typename R, int G, int NT>
static int launch_team(hsweep_s* h, const TeamConfig& cfg, TeamArgs<R>& a) {
  auto kern = sweep_team_kernel<R, G, 0, NT>;
  if (cfg.C > 16) {
    kern = sweep_team_kernel<R, G, 0, NT, true>;   // sibling subtrees of more than 8 CTAs
  } else if constexpr (sizeof(R) == 4 && NT == kThreads) {
    if (a.tc == 1) kern = sweep_team_kernel<R, G, 1, NT>;
    if (a.tc == 2) kern = sweep_team_kernel<R, G, 2, NT>;
  }
  HSW_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem));
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute at[1];
  lc.blockDim = dim3(NT);
  lc.gridDim = dim3(cfg.C * cfg.nteams);
  lc.dynamicSmemBytes = cfg.smem;
  lc.stream = h->stream;
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
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

template <typename R>
static int dispatch_team(hsweep_s* h, const TeamConfig& cfg, TeamArgs<R>& a) {
  if (cfg.nt == kThreads2) {
    switch (cfg.G) {
      case 1: return launch_team<R, 1, kThreads2>(h, cfg, a);
      case 2: return launch_team<R, 2, kThreads2>(h, cfg, a);
      case 4: return launch_team<R, 4, kThreads2>(h, cfg, a);
      case 5: return launch_team<R, 5, kThreads2>(h, cfg, a);
      default: return launch_team<R, 8, kThreads2>(h, cfg, a);
    }
  }
  switch (cfg.G) {
    case 1: return launch_team<R, 1, kThreads>(h, cfg, a);
    case 2: return launch_team<R, 2, kThreads>(h, cfg, a);
    case 4: return launch_team<R, 4, kThreads>(h, cfg, a);
    case 5: return launch_team<R, 5, kThreads>(h, cfg, a);
    default: return launch_team<R, 8, kThreads>(h, cfg, a);
  }
}

static long long al256t(long long x) { return (x + 255) / 256 * 256; }

template <typename R>
static void team_scratch_need(const hsweep_s* h, int nrhs, const TeamConfig& cfg, long long* w_bytes,
                              long long* x_bytes) {
  const long long es = sizeof(Cx<R>);
  *w_bytes = (long long)nrhs * h->N * es;
  *x_bytes = 2LL * cfg.nteams * cfg.C * std::max(1, cfg.dC) * std::max(1, h->rank_max) * cfg.G * es;
}

template <typename R>
static int apply_team_impl(hsweep_s* h, const c128* r, c128* z, int nrhs, bool* used, void* scratch,
                           size_t scratch_bytes) {
  *used = false;
  TeamConfig cfg = choose_team<R>(h, nrhs);
  if (!cfg.ok) return HSWEEP_OK;
  const size_t es = sizeof(Cx<R>);
  long long wb, xb;
  team_scratch_need<R>(h, nrhs, cfg, &wb, &xb);
  void* wptr;
  void* xptr;
  if (scratch) {    // caller-provided scratch: nothing is allocated
    if ((size_t)(al256t(wb) + al256t(xb)) > scratch_bytes) return HSWEEP_ERR_ARG;
    wptr = scratch;
    xptr = (unsigned char*)scratch + al256t(wb);
  } else {
    const long long need_w = (long long)nrhs * h->N;
    if (need_w > h->wcache_cap) {
      int rc = hsw_regrow(h, &h->d_wcache, (size_t)need_w * es);
      if (rc) {
        if (!h->d_wcache) h->wcache_cap = 0;
        return rc;
      }
      h->wcache_cap = need_w;
    }
    const long long need_x = xb / (long long)es;
    if (need_x > h->xch_cap) {
      int rc = hsw_regrow(h, &h->d_xch, (size_t)need_x * es);
      if (rc) {
        if (!h->d_xch) h->xch_cap = 0;
        return rc;
      }
      h->xch_cap = need_x;
    }
    wptr = h->d_wcache;
    xptr = h->d_xch;
  }
  TeamArgs<R> a;
  plan_team<R>(h, cfg.dC, cfg.G, a, cfg.nt);
  a.n = h->n; a.L = h->L; a.leaf = h->leaf; a.nnodes = h->nnodes; a.dC = cfg.dC; a.C = cfg.C;
  a.nteams = cfg.nteams; a.nrhs = nrhs; a.ngroups = (nrhs + cfg.G - 1) / cfg.G;
  a.N = h->N; a.pack_stride = h->pack_stride;
  a.tc = (sizeof(R) == 4 && a.slab_max <= 64 && cfg.nt == kThreads) ? h->opt.sweep_tc : 0;
  a.lo = h->d_lo; a.sz = h->d_sz; a.rank = h->d_rank; a.recoff = h->d_recoff;
  a.pack = reinterpret_cast<const Cx<R>*>(h->d_pack);
  a.north = h->d_north_m; a.r = r; a.z = z;
  a.w = reinterpret_cast<Cx<R>*>(wptr);
  a.xch = reinterpret_cast<typename Tagged<R>::W*>(xptr);
  a.status = h->d_status;
  // test hooks (environment): HSWEEP_TEST_WAIT_LIMIT shortens the waits for other CTAs,
  // HSWEEP_TEST_WITHHOLD=c makes CTA c of the grid never publish its partial sums, so
  // that the CTAs reading them run out of their waits and report HSWEEP_ERR_TIMEOUT
  a.wait_limit = kWaitLimit;
  a.withhold = -1;
  if (const char* e = getenv("HSWEEP_TEST_WAIT_LIMIT")) {
    const long long v = atoll(e);
    if (v > 0 && v < kWaitLimit) a.wait_limit = v;
  }
  if (const char* e = getenv("HSWEEP_TEST_WITHHOLD")) a.withhold = atoi(e);
  const bool prof = h->prof;
  if (scratch) h->prof = false;   // the no-allocation path creates no events
  int rc = HSWEEP_OK;
  // every exchange slot starts with the tag bit set: steps 0 and 1 expect it clear
  if (cudaMemsetAsync(xptr, 0xff, (size_t)xb, h->stream) != cudaSuccess)
    rc = HSWEEP_ERR_CUDA;
  if (rc == HSWEEP_OK) rc = dispatch_team<R>(h, cfg, a);
  h->prof = prof;
  if (rc == HSWEEP_OK) *used = true;
  return rc;
}

static bool team_usable(const hsweep_s* h) {
  return h->pack_valid && !h->slab_bytes_max.empty();
}

}  // namespace

int hsw_team_plan(hsweep_s* h, int nrhs, long long* out) {
  TeamConfig cfg{};
  if (team_usable(h)) cfg = h->prec == HSWEEP_FP64 ? choose_team<double>(h, nrhs) : choose_team<float>(h, nrhs);
  if (!cfg.ok) return 0;
  out[0] = 2; out[1] = cfg.C; out[2] = cfg.G; out[3] = cfg.nteams; out[4] = cfg.nt;
  out[5] = (long long)cfg.smem; out[6] = h->slab_bytes_max[cfg.dC]; out[7] = kKS;
  return 1;
}

int hsw_apply_team(hsweep_s* h, const c128* r, c128* z, int nrhs, bool* used, void* scratch, size_t scratch_bytes) {
  *used = false;
  if (!team_usable(h)) return HSWEEP_OK;
  if (h->prec == HSWEEP_FP64) return apply_team_impl<double>(h, r, z, nrhs, used, scratch, scratch_bytes);
  return apply_team_impl<float>(h, r, z, nrhs, used, scratch, scratch_bytes);
}

size_t hsw_apply_team_scratch_bytes(hsweep_s* h, int nrhs) {
  if (!team_usable(h)) return 0;
  long long wb, xb;
  if (h->prec == HSWEEP_FP64) {
    TeamConfig cfg = choose_team<double>(h, nrhs);
    if (!cfg.ok) return 0;
    team_scratch_need<double>(h, nrhs, cfg, &wb, &xb);
  } else {
    TeamConfig cfg = choose_team<float>(h, nrhs);
    if (!cfg.ok) return 0;
    team_scratch_need<float>(h, nrhs, cfg, &wb, &xb);
  }
  return (size_t)(al256t(wb) + al256t(xb));
}
