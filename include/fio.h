/*
 * fio.h -- C ABI of libfio: GPU apply of the approximate inverse of a discrete Fourier integral
 * operator (FIO), K^{-1} ~ G-dot K-dot*, on one NVIDIA GB300 (sm_103a).
 *
 * The problem (paper section 1, eq. 1.6): u = K f-hat with K_ij = a(x_i, xi_j) exp(2 pi i Phi(x_i, xi_j))
 * on the n^d grids X = {k/n} and Omega = {-n/2 .. n/2-1}^d.  The approximate inverse (section 5,
 * Algorithm 1) is the product of
 *   K-dot*  the adjoint butterfly factorisation (section 2, eq. for K-dot and its adjoint):
 *           L+3 block-sparse factors V_L H_{L-1} ... H_{L/2} D* C*_{L/2} ... C*_{L-1} U_L*;
 *   G-dot   the hierarchical interpolative factorisation of (K*K)^{-1} (section 4, eqs. for G-dot
 *           in 1D and 2D): R_L ... R_1 A_0^{-1} R_1* ... R_L* (2D: R_l Rbar_l pairs).
 * The factors are built once on the host (Python builder) and handed over as one packed buffer.
 *
 * VECTORS.  Every vector argument is a DEVICE pointer to an N x b complex array in column-major
 * order with leading dimension ld >= N (column j = right-hand side j), in natural grid order:
 * 1D index i <-> x_i = i/n (X side) or xi_i = i - n/2 (Omega side); 2D index i1 + n*i2 <-> the
 * point (i1, i2).  Complex values are interleaved (re, im): double pairs for FIO_C128, float
 * pairs for FIO_C64 (the layouts of torch.complex128 / torch.complex64).  Inputs and outputs must
 * not overlap.  b >= 0; b == 0 is a no-op.
 *
 * PRECISION.  FIO_P64 applies the FP64 (complex128) copy of the factors, FIO_P32 the FP32
 * (complex64) copy, which fio_upload_factors derives on the device (FP32 CUDA-core arithmetic).
 * FIO_PTF32 and FIO_PBF16 run the stage products on the tensor cores (tcgen05) with FP32
 * accumulation: TF32 products of the complex64 copy, or products of a bfloat16 copy of the
 * factors with bfloat16-rounded vectors; both take complex64 vectors and are meant as the inner
 * precision of an iterative refinement (their rounding is ~1e-3 resp. ~4e-3 per stage).
 * FIO_PTF32X3 is FP32-accurate on the TF32 tensor cores: each operand value is split into a TF32
 * head and a TF32 tail and a product is summed as head*head + head*tail + tail*head (three MMAs
 * per step, FP32 accumulation; the dropped tail*tail term is ~2^-22 relative); same factors and
 * vectors as FIO_PTF32.  With fewer than 8 right-hand sides the tensor-core precisions fall back
 * to the FP32 CUDA-core kernels.  FIO_PDF takes complex128 vectors and applies a double-float copy
 * of the factors (each FP64 entry as an unevaluated sum of two floats, 48-bit significand) with
 * compensated (twice-working-precision) accumulation on the FP32 CUDA cores: FP64-class results
 * (~1e-14 relative per stage) at the FP32 pipes' rate, for the outer residual of iterative
 * refinement (GB300's FP64 rate is a small fraction of its FP32 rate); it adds two conversion
 * launches per apply and is not accepted by fio_apply_inv_noalloc.  The vector dtype
 * must match the precision (C128 with P64 and PDF, C64 with the others); other pairs return FIO_EINVAL.
 *
 * STREAMS AND SCRATCH.  Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 * default stream) unless stated otherwise.  Each operator owns a scratch pool (device memory for
 * the intermediate stage vectors) that grows on demand; growing synchronises `stream`.  Calls on
 * the same operator must not run concurrently (they share the scratch pool): issue them on one
 * stream.  Distinct operators are independent.
 *
 * ERRORS.  Every call returns an int status: FIO_OK (0) or a negative FIO_E* code; nothing is
 * thrown and nothing aborts.  Launch errors and errors of earlier asynchronous work found at the
 * call return FIO_ECUDA.  fio_strerror gives a static message.  The tensor-core kernels bound
 * every wait; one that gives up sets a per-device flag and leaves its outputs incomplete.  The
 * asynchronous applies cannot see that flag when they return: it is reported (FIO_ETIMEOUT) and
 * cleared by the next synchronising call on the device -- fio_sync, fio_apply_inv_host,
 * fio_solve, fio_apply_profiled, fio_autotune or fio_stage_errors.
 *
 * PACKED FACTOR BUFFER (little-endian; produced by paper_2105_02995_gb300/builder/pack.py):
 *   header, 256 bytes:
 *     0  char[8] magic "FIOPACK1"      8  u32 version (1)     12 u32 d (1 or 2)
 *     16 i64 n                         24 i64 N = n^d
 *     32 u32 n_bf   (butterfly stages, in the order they act on f-hat)
 *     36 u32 n_hif  (HIF stages R_L*, (Rbar_L*), ..., R_1*, (Rbar_1*) in that order)
 *     40 u32 n_root (0 or 1: the stage holding A_0^{-1})      44 u32 flags
 *     48 f64 eps_bf                    56 f64 eps_hif
 *     64 u64 stage_table offset        72 u64 data offset     80 u64 total bytes
 *     88 u64 checksum = sum_k w_k (2k+1) mod 2^64 over the u64 words w_k of [data, total)
 *   stage table: n_bf + n_hif + n_root entries of 64 bytes:
 *     0 u32 kind (0 MAP, 1 INPLACE)  4 u32 nblk  8 u32 R  12 u32 C
 *     16 i64 in_len  24 i64 out_len  32 u64 offset of M  40 u64 offset of in  48 u64 offset of out
 *     56 u32 level   60 u32 role (0 butterfly, 1 HIF cell, 2 HIF edge, 3 root)
 *   per stage: M = complex128[nblk][R][C] (row-major per block), in = int32[nblk][C],
 *   out = int32[nblk][R]; index -1 marks padding; all offsets 256-byte aligned.
 *   MAP stage: y = S x with y[out[b][r]] = sum_c M[b][r][c] x[in[b][c]]; its valid out indices
 *   are a permutation of [0, out_len) and its valid in indices a permutation of [0, in_len).
 *   INPLACE stage (R == C, in == out): x[I_b] <- M_b x[I_b] on disjoint index sets I_b, the
 *   identity elsewhere; in_len == out_len == N.
 *   K-dot = S_{n_bf} ... S_1;  K-dot* = S_1^* ... S_{n_bf}^*;
 *   G-dot = H_1^* ... H_T^* A_0^{-1} H_T ... H_1 (H_t the t-th HIF stage, H_1 = R_L*).
 */
#ifndef FIO_H
#define FIO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FIO_OK 0
#define FIO_EINVAL (-1)      /* bad argument: null pointer, size, ld < N, dtype/precision pair   */
#define FIO_ENOMEM (-2)      /* device (or pinned host) allocation failed                         */
#define FIO_EBADFACTORS (-3) /* packed buffer damaged or inconsistent (magic, sizes, checksum,
                                index lists)                                                      */
#define FIO_ENOCONV (-4)     /* iterative solve stopped at maxit above the tolerance             */
#define FIO_ETIMEOUT (-5)    /* a bounded device wait gave up                                     */
#define FIO_ECUDA (-6)       /* a CUDA runtime call or kernel launch failed                       */
#define FIO_ENOTSUP (-7)     /* the operator lacks the factors this call needs (e.g. no HIF)      */

typedef struct fio_op_s* fio_op;

typedef enum { FIO_C128 = 0, FIO_C64 = 1 } fio_dtype;
typedef enum { FIO_P64 = 0, FIO_P32 = 1, FIO_PTF32 = 2, FIO_PBF16 = 3, FIO_PTF32X3 = 4, FIO_PDF = 5 } fio_precision;
typedef enum { FIO_DIRECT = 0, FIO_PCG = 1, FIO_GMRES = 2, FIO_IR = 3 } fio_method;

#define FIO_MASK_P64 1u
#define FIO_MASK_P32 2u
#define FIO_MASK_TC 4u /* tensor-core copies: block-transposed complex64 and bf16 (both orientations) */
#define FIO_MASK_DF 8u /* double-float copy of the factors (FIO_PDF)                                  */

typedef struct {
  int method;    /* fio_method                                                                 */
  int inner;     /* fio_precision of the preconditioner / inner correction (any fio_precision)  */
  double tol;    /* stop when ||u - K-dot f|| <= tol ||u|| for every right-hand side           */
  int maxit;     /* iteration cap (outer iterations for FIO_IR)                                 */
  int restart;   /* GMRES restart length (FIO_GMRES, and the inner GMRES of FIO_IR)             */
  int outer;     /* fio_precision of the residuals u - K-dot f on complex128 vectors: FIO_P64   */
                 /* (0, FP64 arithmetic) or FIO_PDF (double-float arithmetic)                   */
  fio_op residual_op; /* operator whose K-dot gives the true residuals (NULL: the solved         */
                 /* operator itself); FIO_IR and FIO_DIRECT only.  A butterfly of the same FIO  */
                 /* (same d and n) built with a smaller tolerance: refinement then solves       */
                 /* K-dot_tight f = u, with the loose operator's G-dot K-dot* as the correction */
} fio_solve_opts;

typedef struct {
  int iters;     /* iterations taken                                                            */
  double relres; /* final ||u - K-dot f|| / ||u||                                               */
  int status;    /* FIO_OK or FIO_ENOCONV                                                       */
} fio_solve_info;

/* Validate `packed` (nbytes host bytes; the layout above), copy it to the device of the current
 * CUDA context and derive the precision copies named by precisions_mask (FIO_MASK_P64, FIO_MASK_P32,
 * FIO_MASK_TC (needs P32), FIO_MASK_DF; 0 means all four).  The caller keeps ownership of `packed` and may free it on return
 * (the copy is synchronous with respect to the host).  On success *out owns the device copies
 * until fio_release.  Errors: FIO_EINVAL (null args), FIO_EBADFACTORS, FIO_ENOMEM, FIO_ECUDA. */
int fio_upload_factors(const void* packed, size_t nbytes, unsigned precisions_mask, void* stream,
                       fio_op* out);

/* y = K-dot x: the butterfly factors (section 2, eq. for K-dot), x on Omega, y on X. */
int fio_apply_K(fio_op op, const void* x, void* y, int64_t ld, int b, int dtype, int precision,
                void* stream);

/* y = K-dot* x: conjugate-transposed butterfly factors in reverse order, x on X, y on Omega. */
int fio_apply_Kadj(fio_op op, const void* x, void* y, int64_t ld, int b, int dtype, int precision,
                   void* stream);

/* y = G-dot x ~ (K*K)^{-1} x (section 4, eqs. for G-dot); needs the HIF stages (else ENOTSUP). */
int fio_apply_G(fio_op op, const void* x, void* y, int64_t ld, int b, int dtype, int precision,
                void* stream);

/* f = G-dot K-dot* u ~ K^{-1} u: the direct solver (section 5).  u on X, f on Omega. */
int fio_apply_inv(fio_op op, const void* u, void* f, int64_t ld, int b, int dtype, int precision,
                  void* stream);

/* The DFT F of section 1 and its inverse, for the full solve of u = K F f (f = F^{-1} K^{-1} u):
 *   fio_apply_F     f-hat(xi) = n^{-d} sum_x exp(-2 pi i x.xi) f(x)
 *   fio_apply_Finv  f(x)      =         sum_xi exp(+2 pi i x.xi) f-hat(xi)
 * on the operator's grids (x = k/n, xi = j - n/2 per dimension, 2D index i1 + n*i2), for n a
 * power of two and N = n^d <= 2048^2 (FIO_ENOTSUP otherwise), b <= 65535.  Vectors as for the applies;
 * complex128 in FP64 (FIO_P64) or complex64 in FP32 (FIO_P32).  Batched shared-memory FFT
 * (one pass for 1D N <= 2048, else two: rows and columns in 2D, four-step in 1D). */
int fio_apply_F(fio_op op, const void* f, void* fhat, int64_t ld, int b, int dtype, int precision,
                void* stream);
int fio_apply_Finv(fio_op op, const void* fhat, void* f, int64_t ld, int b, int dtype, int precision,
                   void* stream);

/* As fio_apply_inv, but u and f are HOST pointers (pageable or pinned): the call copies u to the
 * device, applies, copies f back and synchronises `stream` before returning.  FIO_ETIMEOUT when a
 * tensor-core bounded wait gave up (f is then incomplete). */
int fio_apply_inv_host(fio_op op, const void* u_host, void* f_host, int64_t ld, int b, int dtype,
                       int precision, void* stream);

/* Iterative solve of K-dot f = u to ||u - K-dot f|| <= tol ||u|| (section 5, eq. for the CG system):
 *   FIO_DIRECT  f = G-dot K-dot* u (no iteration);
 *   FIO_PCG     CG on K-dot* K-dot f = K-dot* u preconditioned with G-dot (the paper's solver);
 *   FIO_GMRES   GMRES on K-dot f = u right-preconditioned with G-dot K-dot*;
 *   FIO_IR      iterative refinement: residual r = u - K-dot f on complex128 vectors in
 *               opts->outer precision (FP64 or double-float), correction G-dot K-dot* r in
 *               opts->inner precision, FP64 update f += d.
 * Every method computes its true residuals u - K-dot f in opts->outer precision (PCG and GMRES
 * run their Krylov products in FP64 whatever opts->outer is).  With opts->residual_op (FIO_IR,
 * FIO_DIRECT) those residuals, and hence tol and info->relres, refer to that operator's K-dot:
 * the approximate inverse of `op` (section 5) corrects towards the solution of the tighter
 * butterfly, whose distance to the exact K is its own e_a.  An all-zero initial guess is
 * detected and its residual taken as u without an apply.
 * f holds the initial guess on entry (zero it for none) and the solution on return.  dtype must
 * be FIO_C128 (FP64 solution).  info_host (may be NULL) receives one record per right-hand side;
 * the call synchronises `stream`.  Returns FIO_OK, FIO_ENOCONV, or an error code (FIO_EINVAL
 * also for a residual_op of another grid, with another method, or lacking opts->outer's copy). */
int fio_solve(fio_op op, const void* u, void* f, int64_t ld, int b, int dtype,
              const fio_solve_opts* opts, fio_solve_info* info_host, void* stream);

/* Autotuner (batching: the tile shape of every stage launch picked by measurement).  For b
 * right-hand sides in `precision`, time each candidate kernel variant of every stage launch
 * (forward and adjoint, on the operator's own factors and zeroed scratch vectors; best of three
 * launches after one warm-up, each timed launch preceded by a 256 MB write that flushes L2, into
 * a buffer the call allocates and frees) and keep the fastest for that stage, direction, arithmetic type
 * and right-hand-side bucket (b <= 4, 5-8, 9-16, 17-32, > 32).  Later applies of the same type
 * and bucket use the choice; untuned ones keep the built-in choice by b.  Variants: 1..7 tile
 * shapes <TX,TB,TR> of the tiled stage kernel (1 <8,1,2>, 2 <16,1,4>, 3 <16,2,4>, 4 <8,2,2>,
 * 5 <8,4,2>, 6 <32,1,8>, 7 <16,4,4>: TX x TB right-hand sides and 64 rows per 256-thread CTA),
 * 8 the few-right-hand-side kernel (b <= 4), 9 / 10 / 11 complex64 tiles with contiguous
 * per-thread rows and right-hand sides (<16,2,8> on 128 threads, <16,2,4> on 256, <8,4,8> on 128
 * threads and 128-row tiles), 12 variant 11 with every in-place stage (HIF nodes, root) split
 * over its columns into slices summed by a fixed-order reduction, 13 (FP64 and FP32, b >= 5) one
 * warp per block for stages whose padded blocks are at most 32 x 32 (the leaf stages), 14 / 15 /
 * 16 (FP64 and double-float) the tiles of 3 / 6 / 2 with three real products per complex
 * product on the butterfly stages (Gauss's 3M form: the imaginary part's rounding error up to a
 * few times the four-product one; the in-place HIF stages keep four products), 17 (FP32) the
 * tiles of 9 with 16-column chunks, 18 (FP32) the tiles of 11 without their register cap (three
 * CTAs per SM instead of four); with a tensor-core
 * precision and b >= 8: 0 the single-buffer tcgen05 kernel, 20 / 21 / 22 its warp-specialised
 * ring variant with 2 / 3 / 4 chunk stages, 30 the persistent tcgen05 kernel whose factor tiles
 * arrive by TMA (work units of as many 128-row tiles as tensor memory holds, deepest ring), 31
 * the same with every in-place stage (HIF nodes, root) split over its columns into slices summed
 * by a fixed-order reduction (enough work units for the few large blocks of the top levels), 32
 * the TMA kernel with units sized for about eight per SM, 33 the TMA kernel with a six-slot
 * ring, 40 the stage launch on the FP32 CUDA cores with FP32's tuned tile; 0 also for empty
 * stages.  Stages whose rows are not 16-byte aligned (an odd width in a hand-packed buffer) and
 * odd b keep variant 0 or the FP32 CUDA cores.
 * Every variant sums each output's terms in the same order, except 8 (tree reductions), 12 and
 * 31 (the in-place stages' slices) and 14..16 (three products), so results for b >= 5 do not
 * depend on the choice otherwise.  choices (may be NULL when cap == 0) receives
 * the variant per stage launch in stage order, forward before adjoint (the root: forward
 * only); *nchoices (may be NULL) their number.  Synchronises `stream`; must not run
 * concurrently with other calls on the operator. */
int fio_autotune(fio_op op, int b, int precision, void* stream, int* choices, int cap, int* nchoices);

/* Pin the kernel variant of every stage launch of (precision, the bucket of b) to `variant`
 * (0 = the built-in choice): 1..18 as for fio_autotune on the CUDA cores (8 only for b <= 4,
 * 9..12, 17, 18 only for FIO_P32, 13 not for FIO_PDF, 14..16 only for FIO_P64 and FIO_PDF); with a tensor-core precision and b >= 8, 0 (single-buffer kernel),
 * 20, 21, 22 (the warp-specialised ring kernel with 2, 3, 4 chunk stages), 30..33 (the
 * TMA-fed persistent kernel, as for fio_autotune) or 40 (FP32 CUDA cores); a variant that does not apply to a stage
 * (shared memory, alignment, odd b) falls back to 0.  Host-only; FIO_EINVAL for a variant that
 * does not exist for the pair. */
int fio_set_variant(fio_op op, int b, int precision, int variant);

/* Diagnostics: the error of `precision` stage by stage.  Runs the apply `which` (0 K-dot,
 * 1 K-dot*, 2 G-dot, 3 G-dot K-dot*) on x (complex128, device, column-major, ld >= N, b >= 1)
 * twice side by side, in FP64 and in `precision` (FIO_P32, a tensor-core precision or FIO_PDF;
 * x rounded to its vector type), and after every stage launch group (each butterfly stage; each
 * HIF stage and the root) stores ||y_p - y_64|| / ||y_64|| of the intermediate vectors in
 * errs_host[k] (k < cap), in application order; *nerr receives the number of stages.  The FP64
 * path is the one held to 1e-12 of the oracle, so these are errors against the oracle's
 * arithmetic.  Allocates its own work vectors and synchronises `stream`. */
int fio_stage_errors(fio_op op, int which, const void* x, int64_t ld, int b, int precision, void* stream,
                     double* errs_host, int cap, int* nerr);

/* Operator facts: dimension, grid size n, N = n^d, device bytes held (factors + scratch). */
int fio_query(fio_op op, int* d, int64_t* n, int64_t* N, size_t* device_bytes);

/* Stage counts and the number of kernel launches one apply issues (for launch accounting):
 * which = 0 apply_K, 1 apply_Kadj, 2 apply_G, 3 apply_inv. */
int fio_launch_count(fio_op op, int which, int b, int* launches);

/* Diagnostics: the apply `which` (as in fio_launch_count) with a CUDA event recorded on `stream`
 * after every launch group (one butterfly stage; one HIF stage = its compute and copy-back
 * launches; a layout change).  stage_ms[k] (host, cap entries) receives the time of group k in
 * launch order, *nmarks the number of groups.  Synchronises `stream`.  Not for the timed path. */
int fio_apply_profiled(fio_op op, int which, const void* x, void* y, int64_t ld, int b, int dtype,
                       int precision, void* stream, float* stage_ms, int cap, int* nmarks);

/* Size of the static device scratch used by fio_apply_inv_noalloc (64 MiB per device). */
#define FIO_NOALLOC_SCRATCH_BYTES (64u << 20)

/* fio_apply_inv without any device allocation during the call.  (The paper has no counterpart:
 * this entry point exists for callers, not for the method.)
 *
 * Who needs it: code that may not call cudaMalloc while it runs -- for example a caller whose
 * device memory is owned by another allocator (a framework's caching allocator), or a latency-
 * critical loop where the implicit device synchronisation of cudaMalloc/cudaFree is not
 * acceptable.  fio_apply_inv may grow the operator's scratch pool on a larger b; this variant
 * never allocates and never frees: its scratch is a static device array of
 * FIO_NOALLOC_SCRATCH_BYTES that every device loading libfio holds until the process exits.
 *
 * Same arguments, result and errors as fio_apply_inv, plus: FIO_EINVAL when the call needs more
 * scratch than the static array holds (3 work vectors of max_len x b elements, max_len the
 * longest butterfly stage vector; e.g. the 1D N = 256 operator fits any b up to several
 * thousand, the 2D n = 256 operator does not fit at b = 32).  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) and caches it; make that first call
 * before any stream capture.  All calls share the one array, and its contents persist between
 * calls: calls that overlap on the GPU (different streams, threads or operators) race and must
 * be serialised by the caller.  Nothing in the array needs to start at zero. */
int fio_apply_inv_noalloc(fio_op op, const void* u, void* f, int64_t ld, int b, int dtype,
                          int precision, void* stream);

/* Self-test of the bounded device waits (no paper counterpart): launches nblocks CTAs that each
 * wait on an mbarrier nothing arrives at, with a limit of limit_us microseconds (1..1e6).  Every
 * wait must give up and return; *gave_up (host) receives how many did.  Returns FIO_ETIMEOUT when
 * the timeouts were reported as the kernels report them (the expected outcome), FIO_EINVAL for
 * bad arguments, FIO_ECUDA / FIO_ENOMEM otherwise.  Synchronises `stream`; leaves the device
 * usable.  This is how the library's failure path is tested without a device fault or hang. */
int fio_selftest_wait(int limit_us, int nblocks, int* gave_up, void* stream);

/* Measurement utility (no paper counterpart): the device's FP32 FMA throughput, the roofline of
 * the CUDA-core stage kernels.  Times a kernel of independent FMA chains (iters steps of 8
 * chains per thread, 8 CTAs of 256 threads per multiprocessor) with CUDA events on `stream`,
 * best of three launches after one warm-up; *tflops (host) receives 2 x FMAs / time, *ms (may be
 * NULL) that time, *sms (may be NULL) the multiprocessor count.  Synchronises `stream`.
 * FIO_EINVAL for iters outside 1..2^24 or a NULL tflops. */
int fio_probe_fp32(int iters, double* tflops, float* ms, int* sms, void* stream);

/* Synchronise `stream` and report what the asynchronous calls before it left: FIO_ETIMEOUT when a
 * tensor-core bounded wait on the current device gave up since the last synchronising call (the
 * flag is then cleared), FIO_ECUDA when the stream holds a CUDA error, else FIO_OK. */
int fio_sync(void* stream);

/* Free the device copies and scratch of op (synchronises the device first).  NULL is a no-op. */
int fio_release(fio_op op);

/* Static, NUL-terminated description of a status code. */
const char* fio_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* FIO_H */
