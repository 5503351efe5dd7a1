/*
 * amg.h -- C ABI of libamg: the coarse-grid correction of two-level
 * DD-alpha-AMG (Heybrock, Rottmann, Georg, Wettig, "Adaptive algebraic
 * multigrid on SIMD architectures", arXiv:1512.04506) on one GB300 GPU.
 *
 * Operations (paper passages in brackets):
 *   setup      R from per-aggregate Gram-Schmidt and D_c = R D P  [Alg. 5, Eq. cgo, Eq. dagger]
 *   restrict   y_c = R y                                          [Alg. 2, Eq. R; Alg. 6]
 *   apply      y_c = D_c x_c                                      [Alg. 2; Sec. 3 "Application of
 *                                                                  coarse-grid operator"]
 *   prolong    x = P x_c, P = R^dagger                            [Alg. 2]
 *   solve      x_c ~ D_c^{-1} y_c by restarted FGMRES              [Alg. 2, coarse-grid solve]
 *   solve_eo   the same with the even/odd (Schur complement) reduction [Alg. 2, "even/odd
 *              preconditioning" of the coarse solve]
 *   batch_cgc  x = P D_c R y for several lattices in one launch    [Alg. 2; persistent threads of Sec. 3]
 *
 * Conventions (all device buffers are owned by the caller unless stated):
 *   - Fine lattice L = {Lx, Ly, Lz, Lt}, blocks B (B[mu] divides L[mu],
 *     L[mu]/B[mu] >= 2), V = prod L, Vb = prod B, Vc = V / Vb.
 *   - Sites are lexicographic with x fastest; coarse sites likewise.
 *   - Gamma matrices in the chiral basis (gamma_5 = diag(1,1,-1,-1)):
 *     aggregate l = spins {0,1}, aggregate r = spins {2,3} of a block.
 *   - Wilson-clover operator, periodic in all directions:
 *       D psi(x) = (4+m0) psi(x) + C(x) psi(x)
 *                  - 1/2 sum_mu [(1-gamma_mu) U_mu(x) psi(x+mu) + (1+gamma_mu) U_mu(x-mu)^+ psi(x-mu)],
 *       C(x) = csw (i/4) sum_{mu!=nu} sigma_{mu nu} F_{mu nu}(x), F = (Q - Q^+)/8 (clover leaves).
 *   - Complex numbers are interleaved (re, im).  Element types:
 *       AMG_FP64 -> 2 x double, AMG_FP32 -> 2 x float, AMG_BF16 -> 2 x bfloat16.
 *   - Fine vectors: [V][4 spin][3 colour][nrhs]; coarse vectors:
 *     [Vc][2 chirality][ntv][nrhs] (2*ntv components per coarse site, l then r).
 *     Fine vectors have element type vec_prec; coarse vectors are FP64 when
 *     vec_prec is AMG_FP64 and FP32 otherwise.
 *   - Every pointer passed in must be 16-byte aligned.
 *   - All calls are asynchronous on the given stream (a cudaStream_t passed
 *     as void*, NULL = legacy default stream) unless stated.  The returned
 *     status covers argument validation and launch errors; errors detected
 *     on the device (rank deficiency, non-finite values, timeouts) are
 *     reported by amg_sync_status() or by the next synchronising call.
 *   - No C++ exception crosses this interface.  There is no global state.
 */
#ifndef AMG_H
#define AMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AMG_OK = 0,
    AMG_ERR_INVALID_ARG = 1,     /* a size, pointer or precision was rejected           */
    AMG_ERR_UNSUPPORTED = 2,     /* valid request that the library does not implement    */
    AMG_ERR_OOM = 3,             /* device allocation failed                             */
    AMG_ERR_CUDA = 4,            /* a CUDA runtime call or launch failed                 */
    AMG_ERR_TIMEOUT = 5,         /* a bounded device-side wait ran out                   */
    AMG_ERR_RANK_DEFICIENT = 6,  /* Gram-Schmidt norm below 1e-12 |v_j| on an aggregate  */
    AMG_ERR_NONFINITE = 7        /* NaN/Inf met where the checked mode looks for it      */
} amg_status;

typedef enum {
    AMG_FP64 = 0,
    AMG_FP32 = 1,
    AMG_FP16_SCALED = 2,  /* FP16 entries with one FP32 scale per (coarse site, stencil block) */
    AMG_BF16 = 3
} amg_prec;

/* Arithmetic of the Gram-Schmidt and of the D_c = R D P assembly in amg_setup_coarse (the
 * clover field stays FP64). */
typedef enum {
    AMG_SETUP_FP64 = 0,     /* doubles on the FP64 pipe                                      */
    AMG_SETUP_F32PAIR = 1   /* each number an unevaluated sum of two floats (~47 bits), sums by
                               TwoSum and products by the FMA residual, on the FP32 pipes;
                               R and D_c agree with FP64 to about 1e-14 relative; aggregates
                               of more than 1536 entries fall back to the FP64 Gram-Schmidt */
} amg_setup_arith;

typedef struct {
    int L[4];            /* fine lattice extents, mu = 0..3 = x, y, z, t               */
    int B[4];            /* block extents                                              */
    int ntv;             /* number of test vectors N_tv, 1..32, ntv <= 6 Vb            */
    int max_nrhs;        /* largest nrhs later passed to the apply calls (1..64)       */
    double m0;           /* bare mass                                                  */
    double csw;          /* clover coefficient                                         */
    amg_prec link_prec;  /* storage of D_c for apply/solve: FP64, FP32, FP16_SCALED, BF16 */
    amg_prec r_prec;     /* storage of R for restrict/prolong: FP64, FP32, BF16         */
    amg_prec vec_prec;   /* element type of fine vectors: FP64, FP32 or BF16            */
    amg_setup_arith setup_arith;  /* assembly arithmetic; 0 (zero-initialised) = FP64       */
} amg_params;
/* BF16 storage runs on the tensor cores and needs ntv a multiple of 4 and V_block a
 * multiple of 8 (else amg_setup_coarse returns AMG_ERR_UNSUPPORTED); its applies take
 * nrhs = 4, 8, 12 or 16 with FP32 coarse vectors. */

typedef struct amg_coarse *amg_handle;

/*
 * amg_setup_coarse -- Alg. 5 on the GPU, in FP64.
 *   d_U  [V][4 mu][3][3] complex double: U_mu(x), the link from x to x+mu.
 *   d_tv [V][4][3][ntv] complex double: the test vectors v_j (Sec. 2.2).
 * Builds the clover field C from d_U, orthonormalises the test vectors on
 * every aggregate A_i^h by block classical Gram-Schmidt (Sec. 3, "Gram-Schmidt
 * on aggregates"), assembles the self block and the four forward blocks of
 * D_c = R D P (Eq. cgo, Alg. 7; all 2 ntv columns of P at once, as
 * Sec. 3 suggests, in FP64 or, with setup_arith = AMG_SETUP_F32PAIR, in pairs
 * of FP32 numbers) and fills the four backward blocks from
 * Eq. dagger, then stores R and D_c in r_prec / link_prec (Sec. 3: D_c may be
 * kept in half precision).  The handle owns every buffer it allocates; the
 * inputs are read only and may be freed once the call returns.  This call
 * synchronises the stream before returning; it returns
 * AMG_ERR_RANK_DEFICIENT when an aggregate's test vectors are dependent, and
 * then *out is still a valid handle that must be destroyed.
 */
amg_status amg_setup_coarse(const amg_params *p, const void *d_U, const void *d_tv,
                            void *stream, amg_handle *out);

/* y_c = R y [Eq. R, Alg. 6].  d_y: fine vectors, d_yc: coarse vectors. */
amg_status amg_restrict(amg_handle h, const void *d_y, void *d_yc, int nrhs, void *stream);

/* y_c = D_c x_c [Alg. 2]; d_xc and d_yc must not overlap. */
amg_status amg_coarse_apply(amg_handle h, const void *d_xc, void *d_yc, int nrhs, void *stream);

/* x = P x_c with P = R^dagger [Alg. 2]. */
amg_status amg_prolong(amg_handle h, const void *d_xc, void *d_x, int nrhs, void *stream);

/*
 * amg_coarse_solve -- the coarse-grid solve of Alg. 2: restarted FGMRES(m)
 * (classical Gram-Schmidt Arnoldi, Givens rotations) on D_c, started from
 * x_c = 0, until the implicit residual is <= tol ||b|| or max_applies
 * applications of D_c have been made; each right-hand side independently.
 * d_b, d_x: coarse vectors with nrhs right-hand sides.  info (host, may be
 * NULL) receives per RHS {applies, final implicit relative residual} as
 * info[2 r], info[2 r + 1]; passing info synchronises the stream.  To stop
 * at convergence the host follows the device step by step: after queueing
 * application j it waits until Arnoldi step j - 1 has completed, so the call
 * returns shortly after the last step, with the final update of x queued.
 */
amg_status amg_coarse_solve(amg_handle h, const void *d_b, void *d_x, int nrhs, double tol,
                            int restart, int max_applies, void *stream, double *info);

/*
 * amg_coarse_solve_noalloc -- amg_coarse_solve for callers that may not allocate device
 * memory when they solve (a memory manager that forbids allocations outside its pool, a
 * latency path that cannot take cudaMalloc's implicit synchronisation).  The paper has no
 * counterpart; it is a property of this library's interface.  Same arguments and results as
 * amg_coarse_solve, but the Krylov workspace lives in a scratch array compiled into the library
 * (amg_noalloc_scratch_bytes(), 16 MiB, held by every GPU that loads the library until the
 * process exits) and nothing is allocated.  A request whose workspace does not fit is rejected
 * with AMG_ERR_INVALID_ARG (amg_last_error() says by how much).  All calls share the array:
 * calls whose kernels overlap on the GPU race and must be serialised by the caller.  The first
 * call on a device looks up the array's device address (with that device current) and should
 * come before any stream capture.  The address is kept for the life of the process: a
 * cudaDeviceReset (which also invalidates every handle) makes it stale, so a process that resets
 * a device must not call the library on that device again.  Unlike amg_coarse_solve, this call
 * never follows the device from the host to stop early, with or without info: it always
 * launches the whole max_applies budget, and the kernels queued after convergence return at
 * once (they cost launch latency, no work).  With info it then synchronises the stream and
 * reports the applications actually made; without info it does not synchronise.
 */
amg_status amg_coarse_solve_noalloc(amg_handle h, const void *d_b, void *d_x, int nrhs, double tol,
                                    int restart, int max_applies, void *stream, double *info);
/* Size in bytes of the scratch array used by amg_coarse_solve_noalloc. */
size_t amg_noalloc_scratch_bytes(void);

/*
 * amg_coarse_solve_mixed -- the coarse solve to a tight tolerance with a cheap operator, by
 * iterative refinement [Alg. 2's low-precision coarse solve; Sec. 3, half-precision D_c]: each
 * pass solves D_c e = r with FGMRES on h_inner's D_c (FP16 / BF16 storage) to inner_tol, adds e
 * to x_c and recomputes the true residual r = b - D_c x_c with h_outer's D_c (FP32), until
 * |r| <= tol |b| per right-hand side or max_outer passes.  h_outer and h_inner must come from the
 * same lattice, blocks, ntv, links and test vectors; both with FP32 coarse vectors.  info (host,
 * may be NULL) receives per RHS {inner D_c applications, outer passes, final true relative
 * residual} at info[3 r .. 3 r + 2].  Synchronises the stream once per pass.
 */
amg_status amg_coarse_solve_mixed(amg_handle h_outer, amg_handle h_inner, const void *d_b, void *d_x,
                                  int nrhs, double tol, double inner_tol, int restart,
                                  int max_inner_applies, int max_outer, void *stream, double *info);

/*
 * Even/odd-reduced coarse solve [Alg. 2: the coarse system is solved by FGMRES with even/odd
 * preconditioning].  Coarse sites split by parity (x + y + z + t) mod 2; D_c couples only
 * opposite parities off the diagonal, so with the odd half eliminated the coarse system becomes
 *   S x_e = b_e - D_eo D_oo^-1 b_o,   S = D_ee - D_eo D_oo^-1 D_oe,   x_o = D_oo^-1 (b_o - D_oe x_e).
 * Half vectors [Vc/2][2 ntv][nrhs] list the sites of one parity in lexicographic order (site i is
 * entry i / 2 of its half).  Needs every coarse extent L[mu]/B[mu] even, FP64 or FP32 storage of
 * D_c with coarse vectors of the same precision, and nrhs <= min(16, max_nrhs).
 *
 * amg_setup_evenodd -- inverts the self block D_c[i][0] of every odd site (Gauss-Jordan with
 * partial pivoting, FP64) and allocates the half-vector workspace (owned by the handle).
 * Synchronises the stream.  AMG_ERR_UNSUPPORTED for an odd coarse extent or another precision,
 * AMG_ERR_NONFINITE when a self block is singular.  A second call does nothing.
 */
amg_status amg_setup_evenodd(amg_handle h, void *stream);
/* y_e = S x_e on half vectors (d_xe, d_ye: [Vc/2][2 ntv][nrhs], must not overlap). */
amg_status amg_schur_apply(amg_handle h, const void *d_xe, void *d_ye, int nrhs, void *stream);
/*
 * amg_coarse_solve_eo -- D_c x = b for full coarse vectors through the reduction: FGMRES(restart)
 * on S (arguments and info as for amg_coarse_solve; the counts and residuals are those of the
 * reduced system, whose relative residual equals |b - D_c x| / |b_e - D_eo D_oo^-1 b_o|; each
 * application of S streams about the bytes of one application of D_c).
 */
amg_status amg_coarse_solve_eo(amg_handle h, const void *d_b, void *d_x, int nrhs, double tol,
                               int restart, int max_applies, void *stream, double *info);
/* amg_cgc_eo -- x = P x_c with x_c from amg_coarse_solve_eo(R y); arguments as amg_cgc. */
amg_status amg_cgc_eo(amg_handle h, const void *d_y, void *d_x, int nrhs, double tol, int restart,
                      int max_applies, void *stream, double *info);
/* D_oo^-1 in FP64, [Vc/2][2 ntv][2 ntv] row-major by odd half index (synchronises). */
amg_status amg_export_Dinv(amg_handle h, void *out);

/*
 * amg_cgc -- one coarse-grid correction, Alg. 2: x = P FGMRES(D_c, R y).
 * Same arguments as amg_coarse_solve for the solve.
 */
amg_status amg_cgc(amg_handle h, const void *d_y, void *d_x, int nrhs, double tol, int restart,
                   int max_applies, void *stream, double *info);

/* ------------------------------------------------------------------ the two-level method around
 * the coarse-grid correction: fine operator, smoother, V-cycle, outer solve.  They work on fine
 * vectors [V][4][3][nrhs] in vec_prec (FP64 or FP32), nrhs <= max_nrhs, and need amg_setup_fine
 * first (AMG_ERR_UNSUPPORTED otherwise).  The smoother needs every coarse extent L_mu / B_mu even
 * (two block colours) and V_block <= 256 (AMG_ERR_UNSUPPORTED otherwise). */

/*
 * amg_setup_fine -- keeps the links d_U ([V][4][3][3] complex double, device, the array given to
 * amg_setup_coarse; not retained) in the handle in vec_prec, with the clover field of the setup,
 * for the fine operator D.  Asynchronous on the stream; may be called again (replaces the copy).
 */
amg_status amg_setup_fine(amg_handle h, const void *d_U, void *stream);

/*
 * amg_dirac_apply -- out = D psi with the Wilson-clover operator whose block parts Eq. cgo
 * restricts (D = (4 + m0) + C - 1/2 sum_mu [(1 - g_mu) U_mu(x) T_{+mu} + (1 + g_mu) U_mu(x - mu)^dag
 * T_{-mu}], periodic; the clover term C^{ll}, C^{rr} of Alg. 7).  psi and out device, distinct.
 */
amg_status amg_dirac_apply(amg_handle h, const void *d_psi, void *d_out, int nrhs, void *stream);

/*
 * amg_sap -- n_cycles cycles of the domain-decomposition smoother of Alg. 3 on D x = y, in place
 * on x (x is the start and the result): the Schwarz alternating procedure over the aggregation
 * blocks coloured by the parity of their block coordinates, colour 0 then colour 1 in each
 * cycle, each block system B_b e = (y - D x)|_b (B = D without the hops across the block face)
 * solved by n_mr minimal-residual steps from e = 0 and added to x.  y and x device, distinct.
 */
amg_status amg_sap(amg_handle h, const void *d_y, void *d_x, int nrhs, int n_cycles, int n_mr, void *stream);

/* Parameters of the V-cycle: the coarse solve of the coarse-grid correction (FGMRES(coarse_restart)
 * to coarse_tol, at most coarse_max_applies applications of D_c; the paper's tolerance is 0.05) and
 * the smoother (n_smoother SAP cycles of n_mr MR steps per block). */
typedef struct {
  double coarse_tol;
  int coarse_restart;
  int coarse_max_applies;
  int n_smoother;
  int n_mr;
} amg_vcycle_params;

/*
 * amg_vcycle -- one application of the two-level preconditioner of Alg. 1: x = S(y; CGC(y)),
 * the coarse-grid correction of Alg. 2 (as amg_cgc) followed by n_smoother SAP cycles started from
 * it.  y and x device, distinct; x is overwritten.
 */
amg_status amg_vcycle(amg_handle h, const amg_vcycle_params *vp, const void *d_y, void *d_x, int nrhs,
                      void *stream);

/*
 * amg_adaptive_setup -- the adaptive setup of Alg. 4 on this handle.  d_tv ([V][4][3][ntv] complex
 * double, device) holds the random starting test vectors and receives the final ones; d_U is the
 * link field of amg_setup_coarse (complex double, device).  Initial phase: every v_j becomes
 * S_k(v_j; 0) for k = 1, 2, 3 in turn (k SAP cycles on right-hand side v_j from zero, vp->n_mr MR
 * steps per block), R and D_c are rebuilt from them (Alg. 5), and every v_j is divided by its norm.
 * Each of the n_setup passes then replaces every v_j by the V-cycle S(v_j; CGC(v_j)) with the
 * current R and D_c and the parameters vp, and rebuilds R and D_c once all are replaced.  The
 * vectors run through the smoother and the V-cycle in chunks of min(max_nrhs, 16) columns, in the
 * handle's vector precision.  Every copy derived from R and D_c (tensor-core layouts) is rebuilt;
 * even/odd data are dropped (call amg_setup_evenodd again).  Needs amg_setup_fine.  Synchronises
 * the stream.  AMG_ERR_RANK_DEFICIENT if the smoothed vectors lose rank on an aggregate.
 */
amg_status amg_adaptive_setup(amg_handle h, const amg_vcycle_params *vp, const void *d_U, void *d_tv, int n_setup,
                              void *stream);

/*
 * amg_solve -- D u = f by restarted FGMRES(restart) right-preconditioned with the V-cycle (Sec. 1:
 * the two-level method as a preconditioner of a flexible Krylov solver), from u = 0, every
 * right-hand side independently: classical Gram-Schmidt, Givens rotations, stop when the implicit
 * residual is <= tol ||f|| or after max_applies applications of D (each restart after the first
 * recomputes the true residual, one more application).  info (may be NULL): per right-hand side
 * (applications of D, implicit relative residual) as info[2 r], info[2 r + 1].  The scalars are
 * kept on the host, so the call synchronises the stream after every Arnoldi step and at the end.
 * Its Krylov basis and preconditioned vectors (2 restart + 2 fine vectors) are allocated in the
 * handle on first use.  restart <= 64.
 */
amg_status amg_solve(amg_handle h, const amg_vcycle_params *vp, const void *d_f, void *d_u, int nrhs,
                     double tol, int restart, int max_applies, void *stream, double *info);

/* ------------------------------------------------------------------ a third level.  Sec. 3 builds
 * two levels and notes that the method carries over to three, save for a smoother on a coarse
 * grid, which the paper does not have.  Here the coarse lattice is coarsened once more: blocks
 * p2->B of coarse sites, each with two aggregates (the l and r halves of every coarse site's
 * 2 ntv components, so that D_cc keeps the gamma_5 structure of D_c), aggregate dofs enumerated
 * (site in block, lexicographic x fastest; component) slowest first.  R2 holds per aggregate the
 * Gram-Schmidt orthonormalised test vectors (Alg. 5's construction one level down), P2 = R2^dag
 * and D_cc = R2 D_c P2 (Eq. cgo).  The smoother on the coarse grid is n_mr minimal-residual steps
 * on D_c from zero, run as FGMRES(1) (the one-vector case of Alg. 2's solver; each step after the
 * first recomputes the residual, so n_mr steps take 2 n_mr - 1 applications of D_c).  Level-1
 * vectors are coarse vectors of the level-1 handle ([Vc1][2][ntv1][nrhs]), level-2 vectors
 * [Vc2][2][ntv2][nrhs], both in vec_prec. */

/*
 * amg_setup_level2 -- a level-2 handle from the level-1 handle h1 (its D_c) and the level-2 test
 * vectors d_tv2 ([Vc1][2][ntv1][ntv2] complex double, device, not retained).  p2: L = the coarse
 * lattice of h1 (L_mu / B_mu of h1), B = the level-2 blocks (every L_mu / B_mu >= 2), ntv = ntv2
 * <= min(32, ntv1 V_block2), vec_prec = that of h1 (FP64 or FP32) with link_prec and r_prec equal
 * to it, max_nrhs as for any handle.  The result is an ordinary coarse handle for D_cc
 * (amg_coarse_apply, amg_coarse_solve, amg_export_R (R2), amg_export_Dc (D_cc), amg_destroy work on
 * it) plus amg_restrict2 / amg_prolong2; the calls that need a fine lattice (amg_restrict,
 * amg_prolong, amg_cgc, the batch calls, amg_export_clover, amg_setup_fine, amg_setup_evenodd)
 * return AMG_ERR_UNSUPPORTED for it.  Setup in FP64; synchronises the stream.
 * AMG_ERR_RANK_DEFICIENT (handle returned) if the test vectors lose rank on an aggregate.
 */
amg_status amg_setup_level2(amg_handle h1, const amg_params *p2, const void *d_tv2, void *stream,
                            amg_handle *out);

/* amg_restrict2 -- y_cc = R2 y_c (level-1 vector in, level-2 vector out; device, distinct). */
amg_status amg_restrict2(amg_handle h2, const void *d_yc, void *d_ycc, int nrhs, void *stream);

/* amg_prolong2 -- x_c = P2 x_cc (level-2 vector in, level-1 vector out, overwritten). */
amg_status amg_prolong2(amg_handle h2, const void *d_xcc, void *d_xc, int nrhs, void *stream);

/* Parameters of the two-grid cycle on level 1: n_mr minimal-residual steps on D_c before and after
 * the correction (0: none), and the level-2 solve FGMRES(restart) to tol, at most max_applies
 * applications of D_cc. */
typedef struct {
  int n_mr;
  int restart;
  int max_applies;
  double tol;
} amg_level2_params;

/*
 * amg_attach_level2 -- makes h2 (from amg_setup_level2 on h1) the third level of h1: from then on
 * the coarse-grid correction inside amg_vcycle and amg_solve uses one two-grid cycle on level 1
 * (amg_two_grid) in place of the coarse FGMRES (vp's coarse_* fields are then unused), which makes
 * the V-cycle a three-level one.  h2 = NULL detaches.  Destroying either handle detaches them.  lp
 * is copied.  amg_adaptive_setup rebuilds D_c and so refuses (AMG_ERR_INVALID_ARG) while a level 2
 * is attached: detach, run it, then build and attach a new level 2.
 */
amg_status amg_attach_level2(amg_handle h1, amg_handle h2, const amg_level2_params *lp);

/*
 * amg_two_grid -- one two-grid cycle for D_c x_c = y_c on level 1 with the attached level 2:
 * x = MR(y); x += P2 x_cc, x_cc the level-2 FGMRES solution of D_cc x_cc = R2 (y - D_c x);
 * x += MR(y - D_c x).  y_c and x_c device, distinct; x_c overwritten.  Its level-1 and level-2
 * work vectors are allocated in h1 on first use.
 */
amg_status amg_two_grid(amg_handle h1, const void *d_yc, void *d_xc, int nrhs, void *stream);

/*
 * amg_batch_cgc -- x_k = P_k D_ck R_k y_k for n lattices (handles hs[k]) in one
 * persistent launch [Alg. 2's restriction, coarse operator and prolongation; Sec. 3 runs its
 * kernels as persistent threads meeting at synchronisation points rather than fork-join]: each
 * lattice's restriction, one D_c application and its
 * prolongation run as phases separated by per-lattice device barriers with a
 * bounded wait (AMG_ERR_TIMEOUT when a wait runs out).  Each lattice runs in its
 * handle's precision: FP32 R, D_c and vectors (any nrhs), or BF16 R, D_c and fine
 * vectors with nrhs = 4, 8, 12 or 16 (tensor cores; y_c and D_c y_c are kept in
 * the work buffer, y_c as BF16).  Other combinations return AMG_ERR_UNSUPPORTED.
 * The launch is capturable in a CUDA graph.
 * Scratch: the first call for a given set of handles allocates a work buffer
 * owned by hs[0]; later calls reuse it.
 */
amg_status amg_batch_cgc(const amg_handle *hs, int n, const void *const *d_y, void *const *d_x,
                         const int *nrhs, void *stream);   /* n <= 8 */

/*
 * amg_batch_autotune -- (no counterpart in the paper) times the fused batch launch for each
 * candidate shape (1, 2, 3 or 4 CTAs
 * per SM, capped by occupancy, x 2, 3 or 4 bulk-copy ring stages) on the caller's arguments (same
 * as amg_batch_cgc) and keeps the fastest in hs[0] for later amg_batch_cgc calls.  best_ms (may be
 * NULL) receives its time in milliseconds.  Synchronises the stream.
 */
amg_status amg_batch_autotune(const amg_handle *hs, int n, const void *const *d_y, void *const *d_x,
                              const int *nrhs, void *stream, double *best_ms);

/*
 * amg_batch_test_hook -- test hook for the bounded waits of amg_batch_cgc: the next launches whose
 * first handle is h0 expect extra_need more phase-1 jobs for lattice 0 than exist, so its
 * coarse-operator jobs wait until their limit (about one second) runs out; the launch then ends
 * early and amg_sync_status reports AMG_ERR_TIMEOUT.  extra_need = 0 restores normal operation.
 */
amg_status amg_batch_test_hook(amg_handle h0, int extra_need);

/*
 * amg_solve_test_hook -- test hook for the bounded grid barriers of the coarse solve's fused Arnoldi
 * step (1, 2, 4, 8 or 16 right-hand sides): the next solves on h expect extra_arrivals more CTAs at
 * each barrier than exist, so every CTA's wait runs out after its limit (about one second), the
 * step ends early and amg_sync_status reports AMG_ERR_TIMEOUT.  extra_arrivals = 0 restores normal
 * operation.  AMG_ERR_INVALID_ARG for a null handle or a negative count.
 */
amg_status amg_solve_test_hook(amg_handle h, int extra_arrivals);

/*
 * amg_grid_cap_test_hook -- (no counterpart in the paper) test hook for the persistent grid-stride
 * kernels (the bulk-copy and tensor-core restrict / apply / prolong, the even/odd passes and, with h
 * as the first handle, the fused batch): later launches on h use at most max_ctas CTAs, so that a
 * lattice small enough for a whole-array check sends many sites, blocks or jobs through each CTA's
 * copy ring, as the full-size workloads do.  The kernels and their results are unchanged; only the
 * grid is smaller.  max_ctas = 0 restores the occupancy-derived grid (resident CTAs per SM x SMs).
 * AMG_ERR_INVALID_ARG for a null handle or a negative count.
 */
amg_status amg_grid_cap_test_hook(amg_handle h, int max_ctas);

/* R as [Nblock][2][ntv][6 Vb] complex double (row j of R_i^h = v_j^dagger on A_i^h, Alg. 5), device or
 * host out. */
amg_status amg_export_R(amg_handle h, void *out);
/* D_c as [Vc][9][2 ntv][2 ntv] complex double, FP64 as assembled (Eq. cgo, Eq. dagger); directions
 * 0,+x,-x,+y,-y,+z,-z,+t,-t. */
amg_status amg_export_Dc(amg_handle h, void *out);
/* The clover field as [V][2 chirality][6][6] complex double (C^{ll}, C^{rr} of Alg. 7). */
amg_status amg_export_clover(amg_handle h, void *out);
/* D_c as stored for the applies (Sec. 3's half precision, or FP32 / BF16), dequantised to
 * [Vc][9][2 ntv][2 ntv] complex double. */
amg_status amg_export_Dc_stored(amg_handle h, void *out);

/* Per-phase setup times in milliseconds: clover, Gram-Schmidt, assembly, dagger fill+quantise. */
amg_status amg_setup_timings(amg_handle h, double out_ms[4]);

/* Number of kernels this handle has launched so far (a host-side count, for benchmarks). */
amg_status amg_kernel_launches(amg_handle h, unsigned long long *out);

/* Waits for the handle's last stream and reports device-detected errors, then clears them. */
amg_status amg_sync_status(amg_handle h);

amg_status amg_destroy(amg_handle h);
const char *amg_status_string(amg_status s);
/* Text of the last failed CUDA call made by this library on the calling thread ("" if none). */
const char *amg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* AMG_H */
