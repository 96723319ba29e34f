/*
 * hisq.h -- C ABI of the GB300 HISQ staggered Dslash and its even-odd Krylov solvers.
 *
 * The library applies the HISQ Dirac operator of Sec. 5.1 (a one-hop fat-link term X and
 * a three-hop Naik long-link term W in each of the four directions) on one parity of a
 * 4D even-odd lattice, and solves A x = b with A = M^+ M = 4m^2 - D_eo D_oe on even
 * sites (M = 2m + D; Sec. 3.2 "Inverters") by CG, multi-RHS CG and multi-shift CG.
 *
 * Conventions shared by every call
 *   Lattice   dims = {Nx, Ny, Nz, Nt}, each even and >= 4; V = Nx Ny Nz Nt, Vh = V/2.
 *   Canonical site order (Sec. 4.3): index(x) = floor(lex/2) + Vh ((x+y+z+t) mod 2),
 *             lex = x + Nx (y + Ny (z + Nz t)); even sites first.
 *   Links     fat = X, lng = W: complex128 [4][V][3][3], link (mu, x) at index mu*V + index(x),
 *             row-major 3x3, (re, im) interleaved doubles.  By default WITHOUT staggered
 *             phases: the library applies the MILC phases eta_0 = 1, eta_1 = (-1)^x,
 *             eta_2 = (-1)^(x+y), eta_3 = (-1)^(x+y+z) and the antiperiodic time boundary
 *             of the spinors (Sec. 3), unless hisq_opts.links_phased = 1.
 *   Vectors   one parity, complex128 [nrhs][Vh][3] in canonical half-index order.
 *   Streams   `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *             Dslash / normal-operator calls are stream-ordered and asynchronous.  Solver
 *             calls run on an internal stream that first waits for `stream`, synchronise
 *             before returning, and make `stream` wait for their completion.
 *   Errors    every int-returning call returns HISQ_OK (0) or one of the codes below and
 *             records it with a message on the context (hisq_get_last_error,
 *             hisq_last_error_message).  Nothing throws across the ABI.
 *   Memory    the library copies the links at hisq_create and owns that copy; all vectors
 *             passed to calls are owned by the caller and must not alias unless stated.
 */
#ifndef HISQ_H
#define HISQ_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
enum hisq_status {
    HISQ_OK = 0,
    HISQ_EINVAL = 1,        /* invalid argument (dims, pointers, precision, aliasing, ...)   */
    HISQ_ENOMEM = 2,        /* device or pinned-host allocation failed                        */
    HISQ_ECUDA = 3,         /* a CUDA runtime call failed (message holds cudaGetErrorString)  */
    HISQ_ENOTCONVERGED = 4, /* solver reached maxiter or a non-finite residual; x = last iterate */
    HISQ_ETIMEOUT = 5,      /* a bounded device-side wait gave up                             */
    HISQ_EDEVICE = 6,       /* a kernel raised the context's device error flag                */
    HISQ_ENOTBUILT = 7      /* the requested precision / compression was not built at create  */
};

/* ------------------------------------------------------------------ precisions */
enum hisq_prec {
    HISQ_F64 = 0,  /* IEEE double storage, double arithmetic                                   */
    HISQ_F64X = 1, /* double-class: each real stored as an unevaluated float pair (hi + lo,
                      48-bit significand, 8 bytes), float-float arithmetic on the FP32 pipes  */
    HISQ_F32 = 2,  /* float storage and arithmetic                                             */
    HISQ_F16 = 3,  /* half storage (spinors: one float scale per site; links: one float scale
                      per link type), float arithmetic.  As a solver's sloppy precision: half
                      links with FP32 iteration vectors                                       */
    HISQ_BF16 = 4, /* as HISQ_F16 with bfloat16 storage                                        */
    HISQ_NPREC = 5
};

/* ------------------------------------------------------------------ context */
typedef struct hisq_ctx hisq_ctx;

typedef struct {
    int links_on_device;       /* 1: fat/lng are device pointers; 0: host pointers              */
    int links_phased;          /* 1: links already contain eta_mu(x) and the time boundary sign
                                  (on the link whose forward hop wraps); 18-real only           */
    unsigned prec_mask;        /* bit (1u << HISQ_xxx) per storage precision to build;
                                  0 = F64 | F64X | F32 | F16                                    */
    int compression[HISQ_NPREC]; /* 18 (default, also 0) or 12 real numbers per link, per
                                  precision.  12 stores two rows of L/c with c a real constant
                                  per link type such that L/c is in SU(3) (checked at create,
                                  HISQ_EINVAL otherwise) and rebuilds the third row from them  */
    int device;                /* CUDA device ordinal                                            */
    int autotune;              /* 1 (default): time the Dslash launch shapes (right-hand sides
                                  per thread, threads per site) on first use of each precision
                                  and right-hand-side count; 0: size-based defaults             */
} hisq_opts;

/* Fill `opts` with the defaults (host links, unphased, F64|F64X|F32|F16, 18 reals, device 0). */
void hisq_opts_default(hisq_opts *opts);

/* Create a context for one lattice: validates dims (each even, >= 4), copies the links to
 * the device and prepares one internal link store per requested precision (phases folded,
 * compressed, quantised; Sec. 5.1 and the commented compression remark beside it).
 * On error *ctx is NULL.  Links are read, never retained. */
int hisq_create(hisq_ctx **ctx, const int dims[4], const double *fat, const double *lng,
                const hisq_opts *opts);

/* HISQ links from thin gauge links (Sec. 3.1: two levels of smearing, the first with c1 1/8,
 * c3 1/16, c5 1/64, c7 1/384 for the link and its 3-, 5- and 7-link staples, a projection of
 * the result to U(3), the second with c1 1, the same staples, the Lepage term -1/8, and the Naik
 * link (-1/24 + eps_naik/8) W W W of the projected links).  thin: canonical [4][V][3][3]
 * complex128 SU(3) links WITHOUT staggered phases (the layout hisq_create takes); fat, lng:
 * the fat link X and the long (Naik) link in the same layout, ready for hisq_create (the fat
 * link is not unitary: 12-real compression is valid for the long link only).  Host or device
 * buffers (links_on_device), which must not overlap.  FP64 throughout; the U(3) projection is
 * the unitary polar factor (Newton iteration).  Synchronises before returning.  Returns
 * HISQ_EINVAL for bad dims, HISQ_ENOMEM, HISQ_ECUDA, or HISQ_EDEVICE if a first-level link was
 * singular (no projection). */
int hisq_smear_links(const int dims[4], const double *thin, double *fat, double *lng, double eps_naik,
                     int links_on_device, void *stream);

/* Release all device memory of the context.  NULL is accepted. */
void hisq_destroy(hisq_ctx *ctx);

/* Last status recorded on the context (0 if none) and its message (never NULL). */
int hisq_get_last_error(const hisq_ctx *ctx);
const char *hisq_last_error_message(const hisq_ctx *ctx);
const char *hisq_strerror(int status);

/* Geometry queries: half volume and the padded half volume used by internal fields. */
long hisq_half_volume(const hisq_ctx *ctx);

/* ------------------------------------------------------------------ internal-layout fields */
/* A field holds nrhs half-lattice vectors in a precision's internal layout (site-major,
 * 16-byte aligned).  It exists so that reduced-precision operators can be applied and
 * timed without per-call conversions. */
typedef struct hisq_field hisq_field;

int hisq_field_create(hisq_ctx *ctx, int prec, int nrhs, hisq_field **f);
void hisq_field_destroy(hisq_field *f);
/* canonical complex128 [nrhs][Vh][3] (device pointer) <-> internal; stream-ordered */
int hisq_field_import(hisq_field *f, const double *src, void *stream);
int hisq_field_export(const hisq_field *f, double *dst, void *stream);
/* bytes of device memory held by the field */
size_t hisq_field_bytes(const hisq_field *f);

/* ------------------------------------------------------------------ operators */
/* out = D_{p,1-p} in (Sec. 5.1 stencil; p = out_parity).  `in` holds parity 1-p, `out`
 * receives parity p, both canonical complex128 [nrhs][Vh][3] DEVICE buffers that must not
 * overlap.  `prec` selects the link storage and arithmetic of the applied operator; for
 * prec != HISQ_F64 the vectors are converted on the way in (F64X: float pairs; F32, F16,
 * BF16: FP32) and back to double on the way out.  The 16-bit spinor format is applied
 * through hisq_dslash_field.  Returns HISQ_ENOTBUILT if the context lacks that precision.
 * F64X keeps each real as a pair of floats (hi + lo, no per-site scale): its FP64-class
 * accuracy (about 5e-14 relative per site) holds for vector components of magnitude between
 * about 1e-30 and 1e37; below, the low word becomes subnormal and accuracy degrades toward
 * FP32; above, float overflow.  FP64 has the full double range. */
int hisq_dslash(hisq_ctx *ctx, int out_parity, const double *in, double *out, int nrhs, int prec,
                void *stream);

/* out = D_{p,1-p} in on internal fields of the same precision and nrhs (no conversions);
 * the field precision is both the link and the vector precision. */
int hisq_dslash_field(hisq_ctx *ctx, int out_parity, const hisq_field *in, hisq_field *out,
                      void *stream);

/* out = (4 m^2 - D_eo D_oe) in on even sites (A = M^+ M, Sec. 3.2 applyMdaggM);
 * canonical complex128 [nrhs][Vh][3] device buffers on the context's device, no overlap.
 * Like every entry point that launches work, the call makes the context's device current. */
int hisq_mdagm(hisq_ctx *ctx, double m, const double *in, double *out, int nrhs, int prec,
               void *stream);

/* out = (4 m^2 - D_eo D_oe) in in FP64: equal to hisq_mdagm(..., HISQ_F64, ...)'s result up
 * to rounding (the Dslash launch shape may differ, and with it the summation order), but
 * the call allocates no device memory.  The paper has no counterpart: this entry point exists
 * for callers that cannot let a library allocate, such as applications whose device memory
 * belongs to another allocator or a fixed budget, and loops that must not call cudaMalloc
 * or cudaFree because those calls synchronise the whole device.
 * The odd-parity intermediate lives in a fixed device array of 1048576 half-lattice sites
 * (48 MiB) that every GPU loading the library holds until the process exits: nrhs * Vh
 * above 1048576 returns HISQ_EINVAL.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress), so make it before any stream capture.  All calls
 * share the array: calls that can overlap on the GPU (different streams, or other threads)
 * race on it and must be serialised by the caller.  in/out: canonical complex128
 * [nrhs][Vh][3] device buffers on the context's device, no overlap; the call makes the
 * context's device current and is stream-ordered on `stream`. */
int hisq_mdagm_noalloc(hisq_ctx *ctx, double m, const double *in, double *out, int nrhs, void *stream);

/* Fix the Dslash launch shape for (link precision, vector precision, nrhs) instead of the
 * autotuner's choice: n_inner right-hand sides per thread (1, 2, 4, 8; at most 4 for F64 and
 * F64X; must divide nrhs), threads_per_site (1, 2, 4: the four directions are split over
 * that many threads) and site_order, the order in which blocks visit the sites: 0 storage
 * order (t slowest), 1 z and t interchanged (allowed when Nt < Nz and one z-t plane,
 * Nx/2 * Ny sites, is a multiple of 32), -1 the size-based default.  Vector precision equals
 * the link precision, or is HISQ_F32 with 16-bit links.  Results do not depend on the shape
 * beyond the rounding order of the reductions.  Returns HISQ_EINVAL for any other value.
 * The autotuner also searches 64, 128 and 256 threads per block (hisq_tune_set_block),
 * groups of right-hand sides sharing a site (hisq_tune_set_groups) and groups of right-hand
 * sides per block (hisq_tune_set_block_groups). */
int hisq_tune_set(hisq_ctx *ctx, int prec_links, int prec_vectors, int nrhs, int n_inner, int threads_per_site,
                  int site_order);
/* Threads per block (64, 128 or 256; sites per block = threads / threads_per_site) of the shape
 * already stored for the key (by the autotuner or hisq_tune_set, which stores 128); batches of
 * lattices run 128.  HISQ_EINVAL if no shape is stored or the value is not allowed. */
int hisq_tune_set_block(hisq_ctx *ctx, int prec_links, int prec_vectors, int nrhs, int threads_per_block);
/* Groups of right-hand sides per site (1, 2 or 4) of the stored shape: with g > 1, g
 * consecutive threads share one site (threads_per_site must be 1), thread k of them taking
 * right-hand sides k n_inner .. k n_inner + n_inner - 1 of its group of g n_inner, so each link
 * is loaded once for all of them (n_inner <= 4, g n_inner dividing nrhs).  Results do not
 * depend on it beyond the rounding order of the reductions.  HISQ_EINVAL otherwise. */
int hisq_tune_set_groups(hisq_ctx *ctx, int prec_links, int prec_vectors, int nrhs, int rhs_groups);
/* The stored shape for the key: shape = {n_inner, threads_per_site, site_order,
 * threads_per_block, rhs_groups}; HISQ_EINVAL if none is stored yet. */
int hisq_tune_get(const hisq_ctx *ctx, int prec_links, int prec_vectors, int nrhs, int shape[5]);
/* Groups of right-hand sides per block (1, 2 or 4; the N_outer loop of Sec. 5.1 moved into
 * the block) of the stored shape: with g > 1 the block's threads form g slices over the same
 * sites, slice k taking the k-th of the block's g groups of n_inner right-hand sides, and the
 * links are loaded through L1 so that one read from L2 serves all g groups.  Only the plain
 * Dslash uses it (a solver's normal-operator launches keep one group per block); requires
 * threads_per_site 1, n_inner <= 4, rhs_groups 1, at least 32 threads per slice and
 * g n_inner dividing nrhs, else HISQ_EINVAL (also when no shape is stored).  The autotuner
 * searches it.  Results do not depend on it. */
int hisq_tune_set_block_groups(hisq_ctx *ctx, int prec_links, int prec_vectors, int nrhs, int block_groups);
/* The stored shape's groups of right-hand sides per block; HISQ_EINVAL if none is stored. */
int hisq_tune_get_block_groups(const hisq_ctx *ctx, int prec_links, int prec_vectors, int nrhs, int *block_groups);

/* ------------------------------------------------------------------ solvers */
typedef struct {
    double tol;            /* target |b - A x| / |b| (recomputed in FP64), e.g. 1e-10       */
    int maxiter;           /* iteration cap (sloppy iterations)                              */
    int prec_sloppy;       /* precision of the iterated operator and vectors: HISQ_F64 gives
                              plain double CG; F64X/F32/F16/BF16 give mixed precision       */
    int prec_precise;      /* operator of the reliable updates: HISQ_F64 or HISQ_F64X; with
                              F64X the residual that ends the solve is recomputed with the
                              FP64 operator (when built) before the solve is declared done */
    int reliable_interval; /* sloppy iterations between reliable updates (default 100)       */
    double reliable_delta; /* also update when |r| < delta * |r| at the last update (0.1)    */
    int zero_guess;        /* 1: start from x = 0; 0: x holds the initial guess              */
    int host_buffers;      /* 1: b and x are host pointers (copied inside the call)          */
    int check_interval;    /* use_graph = 0: iterations per block of direct launches (50)    */
    int use_graph;         /* 1 (default): iterations run inside a CUDA graph WHILE node
                              that the device stops when every right-hand side pauses or
                              converges; the host looks at the scalars once per phase      */
    int profile;           /* 1: time the sloppy Dslash pair of the second iteration of every
                              phase (graph) or block of check_interval iterations (direct
                              launches) that can run at least three iterations, with CUDA
                              events; the first two iterations of such a phase are launched
                              directly so that the timed launches queue behind the first   */
    int l2_persist;        /* keep the sloppy link field in L2 during the solve (persisting
                              access-policy window on the solver's kernels, within this
                              process's persisting-L2 limit; persisting lines are released
                              when the call returns): 1 on, 0 off, -1 (default) when the
                              whole field fits the device's persisting-L2 maximum          */
    void *stream;          /* cudaStream_t (NULL = legacy default stream)                    */
    int single_reduction;  /* CG: 1: one grid reduction per iteration: the normal operator's
                              epilogue reduces <p,Ap>, |r|^2, <r,Ap>, <Ap,Ap>, and
                              |r'|^2 = |r|^2 - 2 alpha <r,Ap> + alpha^2 <Ap,Ap> gives beta
                              before one pass updates x, r and p (three launches per
                              iteration); 0 (default): the two-reduction form, |r'|^2
                              reduced from the updated r (four launches)                   */
    int persistent;        /* CG with one right-hand side, no shifts and FP32 iteration
                              vectors (sloppy F32, F16 or BF16): run all sloppy iterations
                              between two reliable updates inside ONE cooperatively launched
                              kernel, in the single-reduction arrangement: one block per SM,
                              each owning a range of sites whose x, r, p and Ap stay in
                              shared memory, bounded grid-wide barriers between the steps.
                              Used when the range fits (Vh up to about 2100 sites per SM).
                              -1 (default): when eligible, launch shape 2; 0: never; 1 to 5:
                              when eligible, with that launch shape (threads per block and
                              load scheduling: 1 = 1024, 2 = 512 with the four hops of a
                              direction loaded before their products, 3 = 896, 4 = 1024 and
                              5 = 448 likewise).  A barrier wait that runs out (about 1 s)
                              ends the launch early and the solve returns HISQ_EDEVICE      */
    int selftest_wait;     /* 1: test of that bounded wait: in the first persistent launch one
                              block leaves without arriving at the first barrier, whose wait
                              (bounded to 1 ms here) runs out in every other block; the
                              solve returns HISQ_EDEVICE and the context stays usable      */
} hisq_solve_opts;

typedef struct {
    int iterations;          /* sloppy iterations (max over right-hand sides / shifts)       */
    int reliable_updates;    /* FP64 residual recomputations                                  */
    double true_residual;    /* max over rhs / shifts of |b - A x| / |b|, recomputed          */
    double iterated_residual;/* iterated residual estimate at exit                            */
    double seconds;          /* wall time of the call                                         */
    long dslash_calls;       /* Dslash applications (all precisions)                          */
    double dslash_ms;        /* summed event time of the timed sloppy Dslash launches         */
    long dslash_timed;       /* number of timed launches (profile = 1): dslash_ms / dslash_timed
                                is the average duration of one sloppy Dslash launch          */
    double bytes_moved;      /* algorithmic bytes of the sloppy Dslash applications           */
    long kernels;            /* kernel launches issued by the call (graph nodes included)     */
    double phase_ms;         /* persistent solves with profile = 1: summed event time of the
                                persistent phase launches                                     */
    long phase_iterations;   /* iterations those launches ran: phase_ms / phase_iterations is
                                the time of one sloppy iteration inside the persistent kernel */
    long phase_launches;     /* number of timed persistent launches                           */
    int persistent_ds;       /* launch shape of the persistent kernel (0: not used)           */
} hisq_stats;

void hisq_solve_opts_default(hisq_solve_opts *o);

/* CG on A x_k = b_k for k < nrhs (Sec. 3.2; nrhs > 1 is the multi-RHS variant).
 * b, x: canonical complex128 [nrhs][Vh][3], device buffers unless opts->host_buffers.
 * Returns HISQ_OK once every true residual <= tol, HISQ_ENOTCONVERGED otherwise (x = the
 * last iterate, stats filled).  `residuals` (may be NULL) receives nrhs true residuals. */
int hisq_cg(hisq_ctx *ctx, double m, const double *b, double *x, int nrhs,
            const hisq_solve_opts *opts, hisq_stats *stats, double *residuals);

/* Multi-shift CG: (A + sigma_s) x_s = b for s < nshift, one operator application per
 * iteration on the smallest shift (Sec. 3.2 and its reference to Jegerlehner).
 * sigma_s >= 0 in any order; x[s] are caller-owned [Vh][3] buffers; tol[s] per shift (NULL:
 * opts->tol).  In a reduced sloppy precision every shift is finished by mixed-precision CG
 * from its multi-shift iterate.  `residuals` (may be NULL) receives nshift true residuals. */
int hisq_multishift_cg(hisq_ctx *ctx, double m, int nshift, const double *sigma,
                       const double *b, double *const *x, const double *tol,
                       const hisq_solve_opts *opts, hisq_stats *stats, double *residuals);

/* r(A) b = alpha0 b + sum_s alpha_s (A + sigma_s)^-1 b: a rational function of A applied to b
 * from one multi-shift solve, the way RHMC's pseudofermion heat bath and force use the
 * multi-shift inverter (Sec. 3.2 "Inverters"; the paper prints no coefficients, the caller
 * supplies the partial fractions of its rational approximation).  nterm in 1..64, sigma_s >= 0
 * and finite, alpha_s and alpha0 finite.  Every shifted system is solved to opts->tol (true
 * relative residual, FP64) with opts' precisions; `residuals` (may be NULL) receives the nterm
 * true residuals.  b, x: canonical complex128 [Vh][3] device buffers, no overlap.  The call
 * allocates nterm solution vectors for its duration and synchronises before returning.
 * Returns HISQ_ENOTCONVERGED (x still formed) if a shifted system missed the tolerance. */
int hisq_rational_apply(hisq_ctx *ctx, double m, int nterm, const double *alpha, const double *sigma,
                        double alpha0, const double *b, double *x, const hisq_solve_opts *opts,
                        hisq_stats *stats, double *residuals);

/* Stochastic estimate of the chiral condensate (1/V) Tr M^-1, M = 2m + D (the measurement the
 * paper runs with its CG, Sec. 3): Tr M^-1 = 4m Tr_e A^-1 (D only connects even and odd sites;
 * the odd block of (M M^+)^-1 has the even block's spectrum), and Tr_e A^-1 is estimated by
 * Re <eta_k, A^-1 eta_k> over the caller's noise vectors, solved by multi-RHS CG (up to 64
 * vectors per solve) with opts (zero initial guesses).  eta: device [nnoise][Vh][3] complex128
 * on even sites (Z2 or Gaussian components: unbiased when E[eta eta^+] = 1), nnoise in 1..4096,
 * m > 0.
 * samples (host, may be NULL): the nnoise values Re <eta_k, A^-1 eta_k>; pbp (host, may be
 * NULL): 4 m mean(samples) / V.  Allocates the solutions for the call; synchronises. */
int hisq_condensate(hisq_ctx *ctx, double m, int nnoise, const double *eta, const hisq_solve_opts *opts,
                    double *samples, double *pbp, hisq_stats *stats);

/* Point-source staggered meson correlators along one direction (the hadronic correlation
 * functions with point sources of Sec. 3.3, "along any direction").  G = M^-1 on the three
 * colour point sources at site src = {x, y, z, t}, M = 2m + D on the full lattice, from one
 * three-RHS CG solve of the even-odd system (Sec. 3.2): A x_e = 2m b_e - D_eo b_o,
 * x_o = (b_o - D_oe x_e) / (2m), with opts' precisions and tolerance (zero initial guesses;
 * the FP64 operator must be built: HISQ_ENOTBUILT otherwise).
 * corr (host, required): [8][N_d] doubles, d = direction (0..3 = x, y, z, t),
 *   corr[S][tau] = sum over sites x with (x_d - src_d) mod N_d = tau of
 *                  (-1)^(sum over i in S of (x_{e_i} - src_{e_i})) sum_{a,b} |G_ab(x, src)|^2,
 *   e_0 < e_1 < e_2 the three other directions, bit i of S selecting e_i: the eight local
 *   staggered channels, S = 0 the Goldstone pion.  Slice sums are reduced in a fixed order
 *   (the same inputs give the same bits).
 * prop (device, may be NULL): receives G as complex128 [3][V][3] (source colour, canonical
 *   full-lattice site with the Vh even sites first, sink colour), 16-byte aligned, 144 V bytes.
 * m > 0, src inside the lattice.  Allocates its workspace for the call; synchronises.
 * Returns HISQ_ENOTCONVERGED (corr still formed) if the solve missed the tolerance. */
int hisq_meson_correlators(hisq_ctx *ctx, double m, const int src[4], int direction,
                           const hisq_solve_opts *opts, double *corr, double *prop, hisq_stats *stats);

/* ------------------------------------------------------------------ batches of lattices */
/* Several lattices of different sizes (each its own context, links and mass) in single
 * launches.  The paper runs one lattice at a time and has no counterpart; the Dslash of a
 * batch is the operator of Sec. 5.1 applied to every member at once, the batched solver
 * is the CG of Sec. 3.2 (with the mixed-precision scheme of hisq_cg) run on every member
 * with its own scalars, iterations of all members sharing each launch. */
typedef struct hisq_batch hisq_batch;

/* A batch of n (1..32) contexts on one device.  The batch borrows the contexts, which must
 * outlive it and keep their link stores; a precision is available in the batch when every
 * member built it with the same compression.  Returns HISQ_EINVAL for a bad list. */
int hisq_batch_create(hisq_batch **batch, int n, hisq_ctx *const *ctxs);
void hisq_batch_destroy(hisq_batch *batch);
/* total sites of one parity over the members (the length of packed vectors, in sites) */
long hisq_batch_sites(const hisq_batch *batch);
const char *hisq_batch_last_error_message(hisq_batch *batch);

/* out = D_{out_parity, 1-out_parity} in for every member, one Dslash launch (plus the
 * conversion kernels of a reduced precision).  in/out: packed canonical complex128 device
 * vectors, member k's [Vh_k][3] sites after those of members 0..k-1; no overlap.  Calls on
 * one batch must be serialised by the caller (they share the batch's padded buffers). */
int hisq_batch_dslash(hisq_batch *batch, int out_parity, const double *in, double *out, int prec, void *stream);

/* Solves (4 m_k^2 - D_eo D_oe) x_k = b_k on every member k, as hisq_cg does for one
 * lattice (opts->prec_sloppy, prec_precise, reliable updates, graph); m: n masses (host),
 * b, x: packed canonical device vectors (as for hisq_batch_dslash; host_buffers is not
 * accepted).  `residuals` (may be NULL) receives n true residuals; stats as hisq_cg, over
 * all members.  Returns HISQ_ENOTCONVERGED if any member misses opts->tol. */
int hisq_batch_cg(hisq_batch *batch, const double *m, const double *b, double *x, const hisq_solve_opts *opts,
                  hisq_stats *stats, double *residuals);

/* ------------------------------------------------------------------ learned preconditioner */
/* Not in the paper.  A gauge-covariant parallel-transport network K (layers of complex
 * channel mixing over 17 taps: identity, the 8 one-hop and 8 three-hop transports of the
 * Dslash stencil with the context's phased links) approximates A^-1 and preconditions
 * flexible CG.  Weights: complex, layer l is a [17][C_out][C_in] block, layers concatenated;
 * activations BF16, arithmetic FP32, gradients FP64. */
typedef struct hisq_net hisq_net;

typedef struct {
    int nlayer;            /* layers (default 4); channels 1 -> C -> ... -> C -> 1           */
    int channels;          /* hidden complex channels C: 1, 2, 4 or 8 (default 8)           */
    int link_prec;         /* link store of the transports: HISQ_F16 (default) or HISQ_F32  */
    int epochs;            /* passes over the training pairs (default 4)                    */
    int batch;             /* pairs per Adam step (default 8)                               */
    double lr, beta1, beta2, eps; /* Adam (default 2e-3, 0.9, 0.999, 1e-8)                  */
    double init_hop;       /* scale of the random hopping weights at initialisation (0.05)  */
    unsigned long long seed; /* initialisation and shuffling seed                           */
    int loss;              /* training loss per pair: 0 (default) error norm |K b - x|^2 /
                              |x|^2; 1 residual norm |A (K b - x)|^2 / |b|^2 with
                              A = 4 mass^2 - D_eo D_oe applied with the FP64 links (which the
                              context must hold)                                             */
    double mass;           /* mass of A for loss 1                                           */
    int tensor_cores;      /* 1 (default): the channel mixing of the 8 -> 8 layers runs on the
                              tensor cores (tcgen05, BF16 operands, FP32 accumulation in
                              tensor memory); 0: FP32 arithmetic on the CUDA cores            */
    int selftest_wait;     /* testing only (default 0): every tensor-core layer launch first
                              waits, for about 1 ms, on a barrier that nothing completes, so
                              that the bounded-wait error path runs: the layer's output is not
                              written and the next synchronising call (loss/gradient, train,
                              flexible CG) returns HISQ_EDEVICE                              */
} hisq_net_opts;

void hisq_net_opts_default(hisq_net_opts *opts);
/* Create a network on a context (the context must hold 18-real links of opts->link_prec).
 * Weights start as the identity map plus small random hopping weights.  The network uses
 * the context's link stores: every call but hisq_net_destroy needs the context alive;
 * hisq_net_destroy may run before or after hisq_destroy of the context. */
int hisq_net_create(hisq_ctx *ctx, const hisq_net_opts *opts, hisq_net **net);
void hisq_net_destroy(hisq_net *net);
/* number of complex weights, and host copies of them (interleaved re, im doubles) */
long hisq_net_num_weights(const hisq_net *net);
int hisq_net_get_weights(const hisq_net *net, double *w);
int hisq_net_set_weights(hisq_net *net, const double *w);
/* z = K(b): b, z canonical complex128 [Vh][3] even-site device buffers */
int hisq_net_apply(hisq_net *net, const double *b, double *z, void *stream);
/* loss |K(b) - x|^2 / |x|^2 and its gradient with respect to every weight (host array,
 * interleaved complex, convention dL/dRe + i dL/dIm); b, x device [Vh][3] */
int hisq_net_loss_grad(hisq_net *net, const double *b, const double *x, double *loss, double *grad);
/* Train on npairs (b, x = A^-1 b) pairs, device arrays [npairs][Vh][3]: opts->epochs passes
 * of shuffled mini-batches of opts->batch pairs, Adam.  The last layer's identity weight
 * starts at <b,x>/<b,b> of the first pairs.  losses (may be NULL) receives the mean loss of
 * every epoch. */
int hisq_net_train(hisq_net *net, int npairs, const double *B, const double *X, double *losses);
/* hisq_net_create(ctx, opts) then hisq_net_train on the npairs (b, x = A^-1 b) pairs, in one
 * call: *net receives the trained network (owned by the caller, hisq_net_destroy), or NULL
 * when either step fails, whose status is returned. */
int hisq_precond_train(hisq_ctx *ctx, const hisq_net_opts *opts, int npairs, const double *B, const double *X,
                       hisq_net **net);
/* binary weights with a small header; load creates a network on ctx */
int hisq_net_save(const hisq_net *net, const char *path);
int hisq_net_load(hisq_ctx *ctx, const char *path, hisq_net **net);

/* Flexible CG (inexact-preconditioner CG, Polak-Ribiere beta) on A x = b with z = K(r)
 * (net != NULL) or z = r (net == NULL: reduces to CG):
 *   alpha = conj(<r,z>)/<p,Ap> (<a,b> = sum conj(a) b), x += alpha p, r' = r - alpha Ap,
 *   z' = K(r'), beta = <r' - r, z'>/<r,z>, p = z' + beta p.
 * FP64 vectors; A applied with opts->prec_precise (HISQ_F64 or HISQ_F64X); the final
 * residual is recomputed with the FP64 operator.  b, x: canonical [Vh][3] device buffers.
 * If the network output is not finite or the residual stops decreasing for 50 iterations,
 * the solve continues as plain CG (stats->reliable_updates counts such fallbacks). */
int hisq_fcg(hisq_ctx *ctx, double m, hisq_net *net, const double *b, double *x, const hisq_solve_opts *opts,
             hisq_stats *stats);

/* ------------------------------------------------------------------ domain decomposition */
/* The Dslash on one time slab of a lattice cut into slabs (Sec. 4, "Communication": each
 * sub-lattice keeps its bulk and a halo of the neighbours' boundary sites, exchanged once per
 * operator application).  Slab [t0, t0 + lt) of the global lattice gdims = (Nx, Ny, Nz, Nt),
 * t0 and lt even, lt >= 4, t0 + lt <= Nt.  Fields on the slab use the slab's own even-odd
 * order (Sec. 4.3 on dims Nx, Ny, Nz, lt): [Vh_slab][3] complex128, Vh_slab = Nx Ny Nz lt / 2;
 * a site's parity there equals its global parity.  The stencil reaches three slices across a
 * cut, so D_{p,1-p} on the slab needs the parity 1-p field on the three slices below t0
 * (halo_lo: global t0-3, t0-2, t0-1, modulo Nt) and on t0+lt .. t0+lt+2 (halo_hi): two
 * buffers of 3 F records, F = Nx Ny Nz / 2, slice after slice, the record of (x, y, z) at
 * face index (x + Nx (y + Ny z)) / 2 within its slice.  The slab below sends its three top
 * slices, the slab above its three bottom slices (hisq_dd_pack); moving them between
 * processes or GPUs (NCCL send/recv, a device copy) is the caller's step. */
typedef struct hisq_dd hisq_dd;
/* fat, lng: the GLOBAL canonical [4][V][3][3] links WITHOUT phases (host or device per
 * opts->links_on_device; opts->links_phased must be 0; opts->device selects the GPU).  The
 * library copies the slab's links and the time-direction links of the three slices below
 * it, folds in the MILC phases and the antiperiodic time boundary by global position, and
 * keeps them in FP64; the caller keeps ownership.  Host links are staged on the device for
 * the call (2 x 4 V x 144 bytes, freed before it returns).  HISQ_EINVAL for bad dims or slab
 * bounds. */
int hisq_dd_create(hisq_dd **dd, const int gdims[4], int t0, int lt, const double *fat, const double *lng,
                   const hisq_opts *opts);
void hisq_dd_destroy(hisq_dd *dd);
const char *hisq_dd_last_error_message(const hisq_dd *dd);
/* Vh_slab, and the records of one halo buffer (3 F) */
long hisq_dd_half_volume(const hisq_dd *dd);
long hisq_dd_halo_sites(const hisq_dd *dd);
/* send_lo = the three lowest time slices of `in` (for the slab below), send_hi = the three
 * highest (for the slab above): device buffers of 3 F records, stream-ordered.  With t
 * slowest in the even-odd order each is one contiguous block, copied as such. */
int hisq_dd_pack(hisq_dd *dd, const double *in, double *send_lo, double *send_hi, void *stream);
/* out = D_{p,1-p} in on the slab's sites of parity p = out_parity, FP64, with the time
 * neighbours beyond the slab read from halo_lo / halo_hi.  Device buffers; out must not
 * overlap any input (HISQ_EINVAL). */
int hisq_dd_dslash(hisq_dd *dd, int out_parity, const double *in, const double *halo_lo, const double *halo_hi,
                   double *out, void *stream);

/* ------------------------------------------------------------------ measured roofs */
/* Not part of the paper's method: the ceilings of this GPU that the kernels' timings are
 * compared with, measured on `device` with CUDA events (about 1 s, 2 GB of scratch memory
 * allocated and freed by the call): fused multiply-add throughput in FP32 and FP64 (8 and 16
 * independent chains per thread, 2048 threads per SM, 2 flops per FMA), read bandwidth of
 * 16-byte loads through L2 over 64 MB (L2-resident, the time of an empty launch of the same
 * shape subtracted) and over 2 GB (HBM), the time of one back-to-back launch of an empty
 * kernel, and one grid-wide barrier of the persistent CG kernel (one 512-thread block per
 * SM; -1 if a bounded wait ran out). */
typedef struct {
    double fp32_tflops;
    double fp64_tflops;
    double l2_read_gbs;
    double hbm_read_gbs;
    double launch_us;
    double grid_barrier_us;
} hisq_peaks;
int hisq_measure_peaks(int device, hisq_peaks *out);

#ifdef __cplusplus
}
#endif
#endif /* HISQ_H */
