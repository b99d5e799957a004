/*
 * hsweep: sweeping preconditioner for the 2D Helmholtz equation with the
 * Schur-complement inverses held as hierarchical (H-) matrices, on one GPU.
 *
 * Method: B. Engquist and L. Ying, "Sweeping preconditioner for the Helmholtz
 * equation: hierarchical matrix representation" (2010).
 *   - Section 2.1, Eq. sigma / Eq. helmd: PML stretching and the 5-point matrix A.
 *   - Algorithm 2.5: setup sweep S~_m = A_mm - A_{m,m-1} T~_{m-1} A_{m-1,m},
 *     T~_m = hinv(S~_m), every T~_m held as a weakly admissible H-matrix (Section 2.3),
 *     or in the strongly admissible case with rank R (hsweep_opts.strong_rank).
 *   - Algorithm 2.6: the apply u = M f (forward and backward sweeps of hmatvec).
 *   - Section 2.4: GMRES on M A u = M f.
 *
 * Conventions used by every entry point below.
 *   Grid:    n x n interior nodes p_{i,j} = (i h, j h), h = 1/(n+1), N = n*n.
 *   Vectors: complex128 (hsw_c128), node (i, j) (1-based) at offset (j-1)*n + (i-1),
 *            i.e. row by row with x1 fastest (Section 2.1 ordering).  A batch of
 *            nrhs vectors is [nrhs][N], vector-major.
 *   Memory:  unless stated otherwise, array arguments are DEVICE pointers; the caller
 *            owns them.  The handle owns every internal buffer (factors, scratch).
 *   Streams: all work is enqueued on the stream given to hsweep_setup.  Entry
 *            points that report a result on the host (status codes from the device,
 *            iteration counts, misfit) synchronise that stream before returning.
 *   Errors:  every entry point returns an hsweep status code; on error no output
 *            argument other than the status is guaranteed.  Nothing here calls
 *            exit() or traps the GPU; device-side failures are recorded in a status
 *            word read by hsweep_status.
 *   Threads: a handle may be used by one host thread at a time.
 */
#ifndef HSWEEP_H
#define HSWEEP_H

#include <stdint.h>

#if defined(__GNUC__)
#define HSWEEP_API __attribute__((visibility("default")))
#else
#define HSWEEP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hsweep_s* hsweep_t;
typedef struct { double re, im; } hsw_c128;

/* Status codes. */
enum {
  HSWEEP_OK = 0,
  HSWEEP_ERR_ARG = -1,           /* invalid argument (sizes, null pointers, NaN) */
  HSWEEP_ERR_OOM = -2,           /* a device or host allocation failed; nothing leaked */
  HSWEEP_ERR_CUDA = -3,          /* a CUDA runtime call failed */
  HSWEEP_ERR_NUMERIC = -4,       /* zero pivot or non-finite value on the device */
  HSWEEP_ERR_NOT_CONVERGED = -5, /* GMRES stopped at its iteration cap (best iterate kept) */
  HSWEEP_ERR_TIMEOUT = -6        /* a bounded device-side wait ran out */
};

/* Arithmetic of the H-factors and of the sweeps. */
enum {
  HSWEEP_FP64 = 0,  /* complex128 everywhere */
  HSWEEP_MIXED = 1  /* complex64 H-factors, setup products and sweeps; FP64 leaf
                       inversions, GMRES (Arnoldi orthogonalisation, A-products inside
                       it), residuals and iterative refinement */
};

typedef struct {
  int leaf;          /* maximum leaf size of the cluster tree, 2..8 (default 8) */
  int r_max;         /* rank cap of every factorised block, 1..56 (default 48) */
  int precision;     /* HSWEEP_FP64 or HSWEEP_MIXED (default HSWEEP_MIXED) */
  double pml_C;      /* PML constant C of Eq. sigma (default 2 pi) */
  int pml_form;      /* 0: sigma = (C/eta)((t-eta)/eta)^2 as in Eq. sigma (default);
                        1: sigma = C ((t-eta)/eta)^2 */
  int gmres_max_it;  /* Arnoldi steps per GMRES solve (default 60) */
  int refine_max;    /* outer FP64 refinement steps in HSWEEP_MIXED (default 8) */
  int team;          /* CTAs per sweep team (power of two, 0 = automatic) */
  int groups;        /* right-hand sides per sweep team (1, 2, 4, 5 or 8; 0 = automatic) */
  int sweep_kernel;  /* 0: automatic (default): with strong_rank > 0 the sweep on the strongly
                           admissible format (hsweep_strong_export) where its plan fits, then
                           the bulk-copy-staged sweep on cooperative teams where its
                           shared-memory plan fits, else the basic sweep;
                        1: the basic sweep that reads the factors from global memory;
                        2: the team sweep on the sibling-pair factors (for strong_rank > 0:
                           the stored, recompressed expansion), else the basic sweep */
  int sweep_tc;      /* HSWEEP_MIXED team sweep, ancestor-level contractions: 0 on CUDA cores
                        (default, the faster on GB300); 1 the reductions, 2 the reductions
                        and the expansion, with mma.sync tensor-core instructions (TF32
                        operands in three parts, FP32 accumulation); teams of at most 16 CTAs
                        with slabs of at most 64 rows (ignored otherwise) */
  int sweep_dir;     /* +1 (default): the sweep runs over the layers from x2 = 0 upward
                        (Algorithms 2.5/2.6); -1: from x2 = 1 downward (Section 3.1, the
                        dependence on the sweeping direction).  A downward handle factors
                        the reflected problem (velocity c(x1, 1 - x2)); hsweep_apply, _matvec,
                        _solve and _grad take and return vectors in the caller's orientation
                        (through device scratch of 2 * nrhs * n*n complex128 values, allocated
                        on first use); layer m of hsweep_export_layer / _import_layer /
                        _layer_ranks is the m-th layer of the sweep order; hsweep_apply_noalloc
                        returns HSWEEP_ERR_ARG */
  int pml_sides;     /* bit mask of the sides with a PML: 1 x1 = 0, 2 x1 = 1, 4 x2 = 0, 8 x2 = 1
                        (default 15, all four); a side without one is a Dirichlet boundary
                        (Section 2.5), zero unless data is moved in by hsweep_boundary_rhs.
                        The sweep may start at either kind of side.  When it starts at a side
                        without a PML, the factorisation is built for the operator with a PML
                        of the same width and profile on that side (without absorption the
                        Schur-complement recursion amplifies truncation and rounding errors
                        from layer to layer); hsweep_matvec and the GMRES of hsweep_solve use
                        the true operator, so the solution is that of the stated problem. */
  int strong_rank;   /* 0 (default): weakly admissible H-matrices (siblings are each other's
                        interaction list; Section 2.3).  R = 1..8: the strongly admissible
                        case (Section 2.3; the configuration of the experiments of Section 3,
                        with R = 2): clusters i, i' of one depth are well separated when
                        |i - i'| >= 2, the blocks of the interaction lists have rank at most R
                        (eps_H still truncates below R), neighbouring leaves are dense.  Each
                        T~_m is the rank-R projection, by the randomized SVD with R + 8
                        Gaussian test vectors, of the weakly admissible inverse of S~_m
                        (rank cap r_max); it is written exactly in the sibling-pair factor
                        layout with rank 3 R (L - depth) + leaf at each depth, and r_max is
                        raised to 3 R (L - 1) + leaf when smaller (HSWEEP_ERR_ARG above 56).
                        The setup keeps that layout recompressed to eps_H for its own
                        arithmetic (hsweep_export_layer), and the strongly admissible T~_m
                        exactly in their own format for the sweep (hsweep_strong_export) */
  unsigned rsvd_seed; /* key of the Philox4x32-10 generator of those test vectors (default 0) */
  int team_threads;  /* threads per CTA of the team sweeps (on the sibling-pair factors and on
                        the strongly admissible format): 512 (one CTA per SM), 256 (two CTAs
                        per SM) or 0 (default: the launch plan chooses) */
  int core_kernel;   /* recompression cores C = R_a R_b^t (hsweep_setup_tuning): 0 (default) the
                        setup's autotuned choice, 1 CUDA cores, 2 tensor cores (HSWEEP_MIXED;
                        HSWEEP_FP64 always uses CUDA cores) */
  int krylov_lowp;   /* HSWEEP_MIXED only.  0 (default): every operation of the inner GMRES
                        (Gram-Schmidt dots and updates, norms, scalings, the product with A)
                        computes in FP64.  1: those operations compute in FP32 on the
                        FP64-stored vectors (products and per-thread partial sums in FP32,
                        block and global sums in FP64); the outer residual f - A u, the
                        update u += d and the reported residuals stay FP64.  Faster on GPUs
                        whose FP64 units are slow.  In either arithmetic the inner solve of
                        HSWEEP_MIXED targets at most a relative 4e-6 (the refinement reaches
                        the tolerance). */
} hsweep_opts;

/* Fill *o with the defaults listed above. */
HSWEEP_API int hsweep_default_opts(hsweep_opts* o);

/*
 * The counter-based generator of the randomized SVD's test vectors: Philox4x32-10 (Salmon,
 * Moraes, Dror and Shaw, SC 2011) of the 128-bit counter ctr[4] under the 64-bit key key[2],
 * written to out[4] (host pointers; host computation, no device needed).  The device draws
 * a complex normal pair from the block with counter {row, column pair, block, layer} and
 * key {rsvd_seed, 0x5EED} by the Box-Muller transform.
 * Returns HSWEEP_ERR_ARG on a NULL pointer.
 */
HSWEEP_API int hsweep_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out);

/*
 * The Gaussian test vectors of one well-separated block, as the device draws them (host
 * computation, no device needed): rows x P complex values (P even) column-major in out
 * (host, 2 * rows * P doubles: re, im), entry (row, p) a complex standard normal from the
 * Philox block {row, p / 2, blk, m} under key {seed, 0x5EED} by the Box-Muller transform
 * (the device's sin/cos may differ in the last bits).  Returns HSWEEP_ERR_ARG on bad sizes.
 */
HSWEEP_API int hsweep_rsvd_normals(uint32_t blk, uint32_t m, uint32_t seed, int rows, int P, double* out);

/*
 * The strongly admissible layout of one layer (host computation, no device needed) for n
 * points, leaves of at most `leaf` (2..8) and rank R (1..8); *nfar, *nnear receive the record
 * counts; far ([*nfar][8] ints), near ([*nnear][6] ints) and ranks ([2^(L+1)] ints) are
 * filled when non-NULL (host memory owned by the caller; call once with NULL to size them).
 *   far:  {a, b, ru0, rw0, su, sw, col, l}: the well-separated block of depth l whose rows are
 *         rows ru0 .. ru0+su-1 of node a and whose columns are rows rw0 .. rw0+sw-1 of its
 *         sibling b (heap node numbers, root 1); its rank-R factors occupy columns
 *         col .. col+R-1 of the expanded F_a, F_b
 *   near: {a, b, ca0, na, nb, col}: the dense block of the neighbouring leaves at the corner of
 *         (a, b) (rows ca0 .. ca0+na-1 of a against the first nb rows of b), stored as the
 *         columns [D | I] from col on
 *   ranks: the expanded rank of every node (3 R (L - depth) + nb of its pair; 0 for nodes 0, 1)
 * Returns HSWEEP_ERR_ARG on bad sizes or NULL count pointers.
 */
HSWEEP_API int hsweep_strong_plan(int n, int leaf, int R, int* nfar, int* nnear, int* far, int* near, int* ranks);

/*
 * The strongly admissible T~_m of a handle set up with strong_rank = R > 0 (Section 2.3,
 * the strongly admissible case), in the format its sweep reads.  Leaf j (heap node
 * 2^L + j, s rows; sl, sr rows in the leaves j - 1, j + 1, 0 at the ends of the layer) has
 * its record at entries recoff[j] .. recoff[j + 1] - 1, row i at recoff[j] + i * rstride[j]:
 *     [ T(j, j)[i, :] | T(j, j - 1)[i, :] | T(j, j + 1)[i, :] |
 *       for d = 2..L, t = 0, 1, 2: W_{v_d, t}[i_v, 0..R) ]
 * where v_d is the leaf's ancestor at depth d and i_v the row's index in v_d.  The
 * interaction list of the cluster with index c at depth d (0-based from the left) is
 * (c - 2, c + 2, c + 3) for even c and (c - 3, c - 2, c + 2) for odd c, slot t in that
 * order (partners outside the layer: zero entries); for a well-separated pair,
 * T(u, w) = W_{u, t(w)} W_{w, t(u)}^t.  Every block not listed is zero.
 *   m          layer, 0 <= m < n
 *   records    host, *nentries complex128 values, or NULL
 *   recoff     host, 2^L + 1 entries, or NULL;  rstride: host, 2^L ints, or NULL
 *   nentries   receives the number of entries of one layer, or NULL
 * HSWEEP_ERR_ARG if the handle holds no such records (strong_rank = 0, or a layer was
 * imported since the setup: the apply then uses the team sweep on the sibling-pair factors).
 */
HSWEEP_API int hsweep_strong_export(hsweep_t h, int m, hsw_c128* records, long long* recoff, int* rstride,
                                    long long* nentries);

/*
 * Assemble A for velocity c at angular frequency omega (Eq. sigma, Eq. helmd; PML of
 * width eta = pml_width * h on all four sides) and run the setup sweep of
 * Algorithm 2.5: for m = 1..n, S~_m from T~_{m-1} (hdiagmul + hsub), T~_m = hinv(S~_m).
 * Off-diagonal blocks keep the singular values above eps_H times the block's largest
 * one (at most r_max of them); eps_H = 0 keeps every one up to r_max.
 *   c_dev      device, n*n doubles, node layout as above; every value finite and > 0
 *   omega      > 0;  n >= 3;  0 <= pml_width < n/2;  eps_H >= 0
 *   opt        NULL for the defaults
 *   stream     a cudaStream_t (NULL = the legacy default stream)
 *   out        receives the handle; *out = NULL on error (nothing leaked)
 * Synchronises the stream; returns HSWEEP_ERR_NUMERIC if a leaf pivot vanished.
 */
HSWEEP_API int hsweep_setup(const double* c_dev, double omega, int n, int pml_width, double eps_H,
                 const hsweep_opts* opt, void* stream, hsweep_t* out);

/*
 * Same as hsweep_setup but without the setup sweep: the H-factors are left empty
 * (all ranks 0, zero leaves) for hsweep_import_layer.
 */
HSWEEP_API int hsweep_create(const double* c_dev, double omega, int n, int pml_width, double eps_H,
                  const hsweep_opts* opt, void* stream, hsweep_t* out);

/*
 * z = M r, the approximate inverse of Algorithm 2.6 (forward sweep, reuse of
 * T~_m u_m, backward sweep), for nrhs vectors at once.
 *   r, z  device [nrhs][N]; r is not modified; r and z must not overlap.
 * Stream-ordered; returns after enqueue.
 * CUDA graphs: for an upward handle (sweep_dir = +1) the call enqueues one memset of the
 * exchange slots and one cooperative kernel launch on the handle's stream, and may be
 * captured into a graph on that stream (replays repeat the call on the captured r and
 * z).  A capture allocates nothing: size the handle's buffers first with one call
 * outside the capture with at least as many right-hand sides; a capture that would
 * need larger buffers, or of a downward handle, returns HSWEEP_ERR_ARG.  Once a capture
 * was made, buffers that later calls outgrow are kept until hsweep_free so that the
 * graph's pointers stay valid.  A graph must not be replayed after hsweep_free or after
 * hsweep_import_layer (the captured launch carries the rank tables of the factors as
 * they were), nor concurrently with other work on the handle.
 */
HSWEEP_API int hsweep_apply(hsweep_t h, const hsw_c128* r, hsw_c128* z, int nrhs);

/* y = A x with the 5-point matrix of Eq. helmd (complex128).  x, y device [nrhs][N],
   must not overlap.  Stream-ordered. */
HSWEEP_API int hsweep_matvec(hsweep_t h, const hsw_c128* x, hsw_c128* y, int nrhs);

/*
 * Solve A u = f for nrhs right-hand sides by GMRES on M A u = M f (Section 2.4),
 * unrestarted, x0 = u on entry (pass zeros for the default start).  Each RHS stops
 * when ||M (f - A u)|| <= tol ||M f||.  In HSWEEP_MIXED the preconditioned solve is
 * wrapped in FP64 iterative refinement: every outer step recomputes r = f - A u in FP64
 * and z = M r, stops the RHS when ||z|| <= tol ||M f||, and otherwise runs GMRES on
 * M A d = z and sets u += d (at most refine_max outer steps).  An outer step whose ||z||
 * is at most 5e4 tol ||M f|| and whose inner GMRES reached 0.5 tol ||M f|| ends the loop
 * without another apply: the complex64 sweep departs from a linear map by less than 1e-5
 * relative, so the remaining ||M (f - A u)|| stays below tol ||M f||.
 *   f, u        device [nrhs][N]
 *   iters_out   host int[nrhs] or NULL: Arnoldi steps taken (summed over refinement)
 *   relres_out  host double[nrhs] or NULL: final ||f - A u|| / ||f|| (FP64)
 * Synchronises.  HSWEEP_ERR_NOT_CONVERGED if any RHS missed tol (u holds the best
 * iterate).
 */
HSWEEP_API int hsweep_solve(hsweep_t h, const hsw_c128* f, hsw_c128* u, int nrhs, double tol,
                 int* iters_out, double* relres_out);

/*
 * Misfit J = 1/2 sum_s ||R u_s - d_s||^2 with A u_s = f_s, and its gradient with
 * respect to the velocity c at the handle's c.  R samples the nodes rec_idx.
 * Adjoint: A is complex symmetric (A^t = A), so A^H lambda = b is solved as
 * lambda = conj(A^{-1} conj(b)) with the same factorisation;
 * dJ/dc_i = -2 omega^2 c_i^{-3} sum_s Re(conj(lambda_{s,i}) u_{s,i} / (s1 s2)_i).
 *   f       device [nsrc][N]
 *   rec_idx device int[nrec], node offsets in [0, N)
 *   d       device [nsrc][nrec]
 *   grad    device double[N] (output)
 *   misfit_out host double (output, may be NULL)
 *   tol     GMRES tolerance of the forward and adjoint solves
 * Synchronises.
 */
HSWEEP_API int hsweep_grad(hsweep_t h, const hsw_c128* f, int nsrc, const int* rec_idx, int nrec,
                const hsw_c128* d, double* grad, double* misfit_out, double tol);

/*
 * Non-zero Dirichlet data on one side (Section 2.5, other boundary conditions; e.g. the
 * depth extrapolation problem, u(x1, 1) = b(x1)): f -= (edge coefficient to the boundary)
 * * b on the unknowns next to that side, so that solving A u = f then imposes u = b there.
 * Meaningful on a side without PML (see pml_sides).
 *   side   0: x1 = 0, 1: x1 = 1, 2: x2 = 0, 3: x2 = 1 (the caller's orientation, also for a
 *          downward handle)
 *   b      device, [nrhs][n] complex128, the data along the side in node order
 *   f      device, [nrhs][n*n] complex128, updated in place
 * Stream-ordered on the handle's stream; HSWEEP_ERR_ARG on a bad side or pointer.
 */
HSWEEP_API int hsweep_boundary_rhs(hsweep_t h, int side, const hsw_c128* b, hsw_c128* f, int nrhs);

/* Last device-side error code (an HSWEEP_ERR_* value, 0 if none) and the layer
   (0-based row m) where it was raised, or -1.  Synchronises. */
HSWEEP_API int hsweep_status(hsweep_t h, int* layer_out);

/* Sizes of the handle: fills out[0..7] with n, tree depth L, leaf, r_max,
   precision, number of leaves, total stored factor entries (all layers, actual
   ranks) and bytes per stored entry.  Synchronises. */
HSWEEP_API int hsweep_info(hsweep_t h, long long* out8);

/*
 * Ranks of T~_m (0-based layer m): ranks_out host int[2^(L+1)], entry v (heap order,
 * root = 1, children of v are 2v and 2v+1) is the rank of the factorised block whose
 * left factor sits on node v; entries 0 and 1 are 0.  Synchronises.
 */
HSWEEP_API int hsweep_layer_ranks(hsweep_t h, int m, int* ranks_out);

/*
 * Copy T~_m (0-based layer m) to or from HOST memory, in complex128, in the layout
 * used on the device (weakly admissible, symmetric storage):
 *   leaves  [n_leaves][leaf][leaf], column-major within a leaf (entry (a, b) at
 *           b*leaf + a), zero-padded beyond the leaf's size;
 *   factors for every non-root node v = 2 .. 2^(L+1)-1 in heap order, F_v of size
 *           n_v x r_max column-major (entry (i, k) at k*n_v + i), where n_v is the
 *           node's size and only the first ranks[v] columns are meaningful.  For
 *           siblings a = 2t, b = 2t+1 the off-diagonal blocks are
 *           T(a, b) = F_a F_b^t and T(b, a) = F_b F_a^t; ranks[a] = ranks[b].
 *   ranks   host int[2^(L+1)] as in hsweep_layer_ranks.
 * Buffer sizes: n_leaves*leaf*leaf and sum_v n_v*r_max = n*L*r_max entries.
 * Import converts to the handle's storage precision.  Synchronises.
 */
HSWEEP_API int hsweep_export_layer(hsweep_t h, int m, hsw_c128* leaves, hsw_c128* factors, int* ranks);
HSWEEP_API int hsweep_import_layer(hsweep_t h, int m, const hsw_c128* leaves, const hsw_c128* factors,
                        const int* ranks);

/*
 * Moves the handle to another stream: later work of the handle is enqueued on `stream`
 * (a cudaStream_t; NULL = the legacy default stream), for instance a stream that can be
 * captured into a CUDA graph (the legacy default stream cannot).  Work already enqueued
 * stays where it is; ordering the two streams is the caller's (synchronise the old one,
 * or make the new one wait for it).  HSWEEP_ERR_ARG on a NULL handle.  (A property of
 * the library, not of the method.)
 */
HSWEEP_API int hsweep_set_stream(hsweep_t h, void* stream);

/*
 * Instrumentation.  hsweep_profile(h, 1) brackets every sweep-kernel launch of the
 * apply with a pair of CUDA events on the handle's stream (0 turns it off).
 * hsweep_stats reports, since the last reset: the number of kernels this handle
 * launched (launches), the number of timed sweep launches and their summed
 * device time in milliseconds (sweep_ms).  Any output pointer may be NULL; reset != 0
 * zeroes the counters afterwards.  hsweep_stats synchronises.
 */
HSWEEP_API int hsweep_profile(hsweep_t h, int enable);
HSWEEP_API int hsweep_stats(hsweep_t h, int reset, long long* launches, long long* sweep_launches,
                            double* sweep_ms);

/*
 * The launch plan the apply would use for nrhs right-hand sides (diagnostics):
 * out[0] the sweep kernel (0: basic, 2: bulk-copy-staged on cooperative teams exchanging
 * tagged partial sums, 3: the same on the strongly admissible format; 1 is not used),
 * out[1] CTAs per team, out[2] right-hand sides per team,
 * out[3] teams, out[4] for the basic kernel 1 when its team is the whole grid (a grid barrier),
 * for the team kernels the threads per CTA (512: one CTA per SM, 256: two), out[5] dynamic shared
 * memory per CTA in bytes, out[6] largest per-step factor record of one CTA in bytes,
 * out[7] column slices per row in the expansion (0 for the basic kernel).
 */
HSWEEP_API int hsweep_sweep_plan(hsweep_t h, int nrhs, long long* out8);

/*
 * The setup's autotuning of the recompression cores C = R_a R_b^t (Section 2.3, "Matrix
 * addition": the small matrix whose SVD truncates a block), diagnostics: in complex64 the
 * setup times, on its middle layer, a CUDA-core kernel and a tensor-core kernel (TF32
 * operands in three parts, FP32 accumulation) on the first launch of each kind and keeps
 * the faster.  out6 (host): [0] kind 0 (recompression after a depth step) and [1] kind 1
 * (once per layer): -1 not tuned (complex128, or no launch of that kind), 0 CUDA cores,
 * 1 tensor cores; [2], [3] the two candidates' times (ms) for kind 0; [4], [5] for kind 1.
 */
HSWEEP_API int hsweep_setup_tuning(hsweep_t h, double* out6);

/*
 * z = M r exactly as hsweep_apply, for callers that must not allocate device memory
 * during the call: code running where cudaMalloc is forbidden or unsafe, such as a
 * framework that owns and accounts for all device memory, a latency-critical loop in
 * which cudaMalloc's implicit device synchronisation is not acceptable, or a memory
 * budget that is already fully committed.  (The paper has no counterpart: this is a
 * property of the library, not of the method.)
 *   - Scratch comes from one fixed device array inside the library, of
 *     HSWEEP_NOALLOC_SCRATCH_BYTES bytes (32 MiB), which every GPU that loads the
 *     library reserves until the process exits.  A call whose scratch need
 *     (about nrhs * n*n * 8 bytes in HSWEEP_MIXED, * 16 in HSWEEP_FP64, plus a few MiB)
 *     exceeds it returns HSWEEP_ERR_ARG and does nothing.
 *   - The array's device address is looked up when the handle is created
 *     (hsweep_setup / hsweep_create, on the handle's device) and kept in the handle;
 *     this call makes no lookup.  The current device must be the handle's device.
 *   - Downward handles (sweep_dir = -1) are refused with HSWEEP_ERR_ARG (their apply
 *     needs reflected copies of r and z).
 *   - Every call shares the one array and it keeps the last call's contents; calls
 *     whose GPU work overlaps (other streams, other handles, other threads) race on it.
 *   - r and z are as in hsweep_apply.  No cudaMalloc, cudaFree or allocating library
 *     routine is called.  Stream-ordered; returns after enqueue.
 *   - It may be captured into a CUDA graph on the handle's stream at any time (no
 *     buffers to size first), with the replay rules of hsweep_apply.
 */
#define HSWEEP_NOALLOC_SCRATCH_BYTES (32u << 20)
HSWEEP_API int hsweep_apply_noalloc(hsweep_t h, const hsw_c128* r, hsw_c128* z, int nrhs);

/* Release every resource of the handle (NULL is allowed). */
HSWEEP_API void hsweep_free(hsweep_t h);

#ifdef __cplusplus
}
#endif
#endif /* HSWEEP_H */
