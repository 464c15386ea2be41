/*
 * sht.h -- C ABI of the GB300 butterfly spherical harmonic transform.
 *
 * Method: M. Tygert, "Fast algorithms for spherical harmonic expansions, III".
 * The library applies the associated-Legendre stage of the spherical
 * harmonic transform (the sums over k of Section 2, eq. alternate_expansion)
 * through a precomputed multilevel butterfly of interpolative decompositions
 * (Section 2.1 Lemma interpolation_lemma / Remark QR_algorithm; Section 2.2
 * eqs. 1-6, top, bottom; Section 3 depth-first precomputation), per order m,
 * with the even/odd parity split of Section 2.3 taken from the symmetric
 * Gauss-Legendre nodes (Section 2, eq. thetas).  The transposed application
 * (Section 2.2, remark after Figure multi) gives the analysis direction.
 *
 * Conventions shared by every entry point:
 *   - l is the bandlimit parameter: degrees k = 0..2l-1, orders m = 0..2l-1
 *     (Section 2, eq. expansion); the grid has 2l Gauss-Legendre nodes
 *     x_0 < ... < x_{2l-1} (zeros of P-bar^0_{2l}) and 4l-1 equispaced
 *     phi_j = 2 pi (j + 1/2) / (4l - 1) (eq. phis).
 *   - P-bar^m_k is the normalized associated Legendre function of Section 2.3,
 *     eq. association (orthonormal on (-1,1), no Condon-Shortley sign).
 *   - beta (coefficients): a REAL field is assumed, so only m >= 0 is stored;
 *     beta^{-m}_k = conj(beta^m_k) and beta^0_k is real.  Storage is an
 *     m-major triangle of complex numbers (interleaved re, im):
 *     beta^m_k at index offset(m) + (k - m), offset(m) = sum_{m'<m} (2l - m'),
 *     k = m..2l-1; 2l(2l+1)/2 entries.
 *   - G (Legendre-stage values): G^m(x_i) = sum_{k=m}^{2l-1} beta^m_k
 *     P-bar^m_k(x_i), a [2l][2l] complex array, row m, column i (nodes
 *     ascending).
 *   - values (grid): real f(theta_i, phi_j), a [2l][4l-1] array, row i
 *     (cos(theta_i) = x_i ascending), column j.
 *   - Precision selects the factor format and arithmetic:
 *       SHT_FP64    float64 factors, float64 arithmetic; complex128 beta/G,
 *                   float64 values.
 *       SHT_SPLIT32 factors stored as hi/lo float32 pairs (hi = fl32(a),
 *                   lo = fl32(a - hi)) applied with compensated (double-float)
 *                   float32 arithmetic; same I/O types as SHT_FP64.
 *       SHT_FP32    float32 factors and arithmetic; complex64 beta/G,
 *                   float32 values.
 *       SHT_SPLIT32_ACC64  the SHT_SPLIT32 factors, products formed as
 *                   float32 error-free pairs (as SHT_SPLIT32) but summed in
 *                   float64 (the high parts) and float32 (the low parts);
 *                   same I/O types as SHT_FP64.  It shares the SHT_SPLIT32
 *                   streams (sht_prepare of either builds both).
 *   - All device pointers are caller-owned, must be 16-byte aligned
 *     (8-byte for SHT_FP32), and are only read/written asynchronously on the
 *     given stream.  Entry points never synchronize the stream unless stated.
 *   - Errors are returned as sht_status; nothing aborts or throws.  Argument
 *     checks happen on the host before any launch; a failed check launches
 *     nothing and leaves outputs untouched.
 */
#ifndef SHT_H
#define SHT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sht_plan_s* sht_plan_t;
/* Same object as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* sht_stream_t;

typedef enum {
  SHT_FP64 = 0,
  SHT_FP32 = 1,
  SHT_SPLIT32 = 2,
  SHT_SPLIT32_ACC64 = 3
} sht_precision;

typedef enum {
  SHT_OK = 0,
  SHT_ERR_INVALID_ARG = 1,   /* bad size, NULL pointer, misaligned pointer */
  SHT_ERR_OOM = 2,           /* host or device allocation failed */
  SHT_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  SHT_ERR_PLAN_CORRUPT = 4,  /* plan file truncated, wrong version, bad checksum */
  SHT_ERR_TIMEOUT = 5,       /* a bounded device wait gave up (see sht_last_device_status) */
  SHT_ERR_UNSUPPORTED = 6,   /* e.g. a compute call on a host-only plan */
  SHT_ERR_NO_DEVICE = 7      /* no CUDA device is visible */
} sht_status;

/* Human-readable name of a status code (static string, never NULL). */
const char* sht_status_string(sht_status s);

/* Text of the last CUDA or cuFFT failure seen by an entry point on the
 * calling thread ("" if none); valid until the next call on this thread. */
const char* sht_last_error_detail(void);

/* ------------------------------------------------------------------ plans */

typedef struct {
  /* Leaf width C of the first butterfly level (Section 2.2: blocks of
   * n x floor(C) columns; Section 5 uses C = 60).  Default 64. */
  int leaf_cols;
  /* Rows i of unit (m, p) whose weighted row norm ||A_{i,:}||_2 is below
   * trim_eps / sqrt(l) are dropped (output 0 there); the dropped rows'
   * total Frobenius norm is <= trim_eps.  < 0 selects eps_id; 0 disables. */
  double trim_eps;
  /* A butterfly level is only added while every row band keeps at least
   * this many rows.  Default leaf_cols / 2. */
  int min_band_rows;
  /* 1: build the factorization on the host only (no CUDA calls at all);
   * compute entry points then return SHT_ERR_UNSUPPORTED.  Used by
   * host-side tests and tools. */
  int host_only;
  /* Host threads for the precomputation; 0 = all hardware threads. */
  int num_threads;
  /* Bytes of one record chunk: a consumer warp fetches its op records
   * (headers, wait lists, index lists) in chunks of this size into a ring of
   * two (a power of two, 512..4096; 0 = default 1024).  A tuning knob. */
  int page_bytes;
  /* eps used for the IDs of the SHT_FP32 factors; <= 0 selects
   * max(eps_id, 1e-7).  (FP32 cannot use ranks below its own precision.) */
  double eps_fp32;
  /* Warps per CTA of the sweep kernels (8, 12 or 16; 0 = 16).  The planner
   * schedules every op of a work item onto one of these warps (list
   * scheduling over the item's dependency graph), so the factor streams are
   * built for this count.  A tuning knob; results do not depend on it. */
  int consumer_warps;
  /* Must be 0: op values always travel apart from the records, in a value
   * region from which each warp bulk-copies its next op's block into a
   * staging slot.  Other values are refused (SHT_ERR_INVALID_ARG). */
  int values_inline;
  /* Tests of failure detection only (default 0): 1 makes the first compute
   * op of the first order of every stream list itself as its predecessor, a
   * completion that never comes.  Launches of such a plan end when the
   * kernel's bounded wait gives up (about 2 s): every wait of the CTA
   * returns, copies in flight are drained, and sht_last_device_status
   * reports SHT_ERR_TIMEOUT; the context stays usable. */
  int debug_unmet_dependency;
  /* Values kept apart: the most values one op may hold, which is the size of
   * a consumer warp's staging slot (a multiple of 32 in 128..2048; 0 = one
   * 8 KB slot's worth: 1024 values for SHT_FP64 and the split formats, 2048
   * for SHT_FP32).  Smaller slots let more consumer warps fit in shared
   * memory, at the cost of splitting blocks into more ops.  A tuning knob. */
  int slot_values;
  /* 1: compute the factorizations (column generation, IDs, depth-first
   * merges of Section 3) on the plan's GPU, one CTA per parity block,
   * instead of on host threads; the host still lays out and encodes the
   * streams.  The columns are the host builder's bit for bit; ranks can
   * differ where a residual norm sits at eps_id, since the QR rounds in
   * another order.  Needs host_only = 0.  Default 0. */
  int device_build;
  /* Device build only: the most device memory, in MB, for the records the
   * GPU writes back (0 = automatic: half the dense operator, at most a
   * quarter of the free memory).  Blocks that do not fit are built again in
   * further launches, each ending with the same streams; a budget too small
   * for the largest single block fails with SHT_ERR_INVALID_ARG. */
  int device_build_arena_mb;
  /* Path of a plan file used as a cache (NULL: none).  When the file exists,
   * is intact and was made with the same l, eps_id, leaf_cols, trim and band
   * options, the plan reads its factorizations from it instead of computing
   * them (see sht_plan_load); otherwise it computes them and writes the file
   * (sht_plan_save), replacing a stale or corrupt one (the reason is left in
   * sht_last_error_detail).  A failed write fails plan creation with
   * SHT_ERR_INVALID_ARG.  The string is read during the call only. */
  const char* plan_cache;
  /* Staging slots per consumer warp: 0 or 1 (one 8 KB slot; the copy of a
   * warp's next op starts as soon as its current op has read the slot).
   * Other values are refused (SHT_ERR_INVALID_ARG). */
  int staging_slots;
} sht_plan_opts;

typedef struct {
  int l;
  double eps_id;
  int leaf_cols;
  int n_units;           /* orders m = 0..2l-1 */
  int n_blocks;          /* IDs in all butterflies (both parities, all m) */
  int k_max;             /* max ID rank (Section 5 tables: k_max) */
  double k_avg;          /* mean ID rank (k_avg) */
  double k_sigma;        /* std. deviation of ID ranks (k_sigma) */
  double max_abs_T;      /* largest |entry| of any interpolation matrix (Remark QR_algorithm bound: 2) */
  int max_levels;        /* deepest butterfly (number of merge levels) */
  int n_direct_units;    /* (m, p) blocks stored dense because compression did not pay */
  long long rows_total;  /* sum over (m, p) of l */
  long long rows_kept;   /* sum over (m, p) of kept rows after trimming */
  long long dense_values;    /* sum over (m, p) of l * n_{m,p}: the dense operator */
  long long factor_values;   /* stored factor values (one direction, eps_id factors) */
  long long index_bytes;     /* skeleton/redundant index bytes (one direction) */
  long long stream_bytes_fp64;   /* device bytes streamed per transform, per direction */
  long long stream_bytes_split32;
  long long stream_bytes_fp32;
  long long factor_values_fp32;  /* stored factor values of the eps_fp32 factorization */
  double t_quad;         /* seconds: Gauss-Legendre nodes and weights */
  double t_comp;         /* seconds: columns + IDs + butterflies (host threads, or the GPU
                          * with device_build) and stream encoding */
  double t_upload;       /* seconds: device upload of the prepared precisions */
  long long m_max_words; /* peak float64 words held by one unit's depth-first build */
  int smem_bytes;        /* dynamic shared memory of the sweep kernels */
  int page_bytes;        /* bytes per record chunk (the value in effect) */
  double t_factor;       /* seconds of t_comp spent on the factorizations (the rest encodes
                          * the streams) */
  double t_factor_kernel; /* seconds of t_factor in the device builder's kernels (0 for a
                           * host build) */
  double factor_flops;   /* floating-point operations the float64 IDs need (Section 2.1,
                          * Remark QR_algorithm): per block of h rows, w columns and rank k,
                          * sum over steps i < k of 4 (h - i - 1)(w - i - 1) for applying
                          * the reflector, plus k^2 (w - k) for T = R11^{-1} R12 */
  long long id_swaps;    /* skeleton/redundant exchanges of the strong rank-revealing step
                          * (Remark QR_algorithm: coefficients at most 2), float64 IDs */
} sht_plan_stats_t;

/* Fills *opts with the defaults listed above. */
sht_status sht_plan_opts_default(sht_plan_opts* opts);

/* Builds the plan for bandlimit l (1 <= l <= 1024) and ID precision eps_id
 * (0 < eps_id < 1): Gauss-Legendre nodes, the parity-split weighted Legendre
 * blocks A^{m,p}_{ij} = sqrt(2 w_{l+i}) P-bar^m_{m+p+2j}(x_{l+i}) (the GL form
 * of Section 4, eqs. transform/transform2) generated column by column with
 * the x^2 recurrence of Section 2.3 (eqs. c_rec, d_rec, recurrence0,
 * recurrence) with exponent tracking, compressed by the depth-first
 * butterfly of Section 3.  The FP64 factor streams are built and (unless
 * host_only) uploaded; other precisions are built at first use or by
 * sht_prepare.  *out receives the plan, or NULL on error.  Allocates host
 * and device memory owned by the plan. */
sht_status sht_plan_create(int l, double eps_id, sht_plan_t* out);
sht_status sht_plan_create_ex(int l, double eps_id, const sht_plan_opts* opts, sht_plan_t* out);

/* Frees the plan and all memory it owns.  NULL is a no-op.  The caller must
 * ensure no work using the plan is still in flight. */
sht_status sht_plan_destroy(sht_plan_t plan);

/* Copies the plan statistics into *out: the rank statistics, costs and
 * errors the paper tabulates (Section 5, k_max, k_avg, k_sigma, t_quad,
 * t_comp, m_max) plus the stream sizes of every precision.
 * sht_plan_stats is the same call under its shorter name. */
sht_status sht_plan_get_stats(sht_plan_t plan, sht_plan_stats_t* out);
sht_status sht_plan_stats(sht_plan_t plan, sht_plan_stats_t* out);

/* Builds (host) and uploads (device) the factor streams of one precision.
 * Synchronous.  Idempotent. */
sht_status sht_prepare(sht_plan_t plan, sht_precision prec);

/* Plan files.  The precomputation (Sections 3 and 4: columns, IDs,
 * depth-first merges) dominates a plan's cold start, so a plan's
 * factorizations can be kept on disk.  A plan file holds a versioned header
 * with the options the factorizations were computed with, a table of
 * per-block offsets and checksums, and the factorizations (float64, and
 * float32 if that precision was prepared).  Factor streams are not stored:
 * they are re-encoded on load for the caller's page size and value cap. */

/* Writes the plan's factorizations to path (through a temporary file renamed
 * into place).  Synchronous; SHT_ERR_INVALID_ARG with a detail on I/O
 * errors. */
sht_status sht_plan_save(sht_plan_t plan, const char* path);

/* Creates a plan from a plan file: l, eps_id and the factorization options
 * (leaf_cols, trim_eps, min_band_rows, eps_fp32) come from the file, the
 * other options (page_bytes, host_only, consumer_warps, ...) from opts (NULL:
 * defaults).  The streams are then encoded and uploaded as by
 * sht_plan_create_ex.  SHT_ERR_INVALID_ARG if the file cannot be opened;
 * SHT_ERR_PLAN_CORRUPT if it is truncated, of another format version, or a
 * checksum or size does not match. */
sht_status sht_plan_load(const char* path, const sht_plan_opts* opts, sht_plan_t* out);

/* The plan's Gauss-Legendre nodes x[2l] (ascending) and weights w[2l] (host
 * arrays owned by the caller). */
sht_status sht_plan_nodes(sht_plan_t plan, double* x, double* w);

/* Host copy of the factor stream of one precision and direction (0 =
 * synthesis, 1 = analysis), for inspection and host-side verification: the
 * record region (the scheduled work items) followed by the value region
 * (layout documented in paper_0910_5435_gb300/csrc/sht_stream.h).  *bytes
 * receives the total and *page_bytes_total (if not NULL) the size of the
 * record region.  With dst == NULL only the sizes are set. */
sht_status sht_plan_stream(sht_plan_t plan, sht_precision prec, int direction,
                           void* dst, size_t* bytes, size_t* page_bytes_total);

/* ----------------------------------------------- Legendre stage (hot path) */

/* Every launch of a plan uses one work-queue counter per (precision,
 * direction): launches of the same plan, precision and direction must not
 * overlap in time (use one stream per plan, or one plan per stream).
 * Launches of different plans, precisions or directions may overlap. */

/* Synthesis: G^m(x_i) = sum_{k=m}^{2l-1} beta^m_k P-bar^m_k(x_i) for all m and
 * all 2l nodes (Section 2, eq. alternate_expansion, the sums over k), through
 * the butterfly (Section 2.2) of each parity block, followed by the parity
 * unfold G(x_{l+i}) = E_i + O_i, G(x_{l-1-i}) = E_i - O_i (Section 2.3).
 * beta: device, triangle layout (complex128, or complex64 for SHT_FP32).
 * G:    device, [2l][2l] complex.  Asynchronous on stream. */
sht_status sht_legendre_synthesize(sht_plan_t plan, sht_precision prec,
                                   const void* beta, void* G, sht_stream_t stream);

/* Analysis: beta^m_k = sum_{i=0}^{2l-1} w_i P-bar^m_k(x_i) G^m(x_i) (the
 * Gauss-Legendre quadrature that inverts synthesis on band-limited data),
 * applied as the transposed butterfly (Section 2.2, remark after Figure
 * multi; Section 4: the per-order maps are unitary, so the inverse is the
 * transpose).  G: device [2l][2l] complex; beta: device triangle. */
sht_status sht_legendre_analyze(sht_plan_t plan, sht_precision prec,
                                const void* G, void* beta, sht_stream_t stream);

/* Adjoint of synthesis (no quadrature weights): beta-hat^m_k =
 * sum_i P-bar^m_k(x_i) G-hat^m(x_i).  Same layouts as analysis.  Used as the
 * backward pass of synthesis. */
sht_status sht_legendre_synthesize_adjoint(sht_plan_t plan, sht_precision prec,
                                           const void* G, void* beta, sht_stream_t stream);

/* Device status word of the plan's last launches: SHT_OK, or SHT_ERR_TIMEOUT
 * if a bounded wait inside a kernel gave up (the kernel then stopped early
 * and its outputs are undefined).  Synchronizes the stream, then clears the
 * word. */
sht_status sht_last_device_status(sht_plan_t plan, sht_stream_t stream);

/* ---------------------------------------------- phi stage and full SHT */

/* Bytes of the caller-provided workspace of the entry points below for this
 * precision: one [2l][2l] complex array (16 bytes per entry, 8 for
 * SHT_FP32). */
size_t sht_workspace_bytes(sht_plan_t plan, sht_precision prec);

/* Sums over m of Section 2, eq. alternate_expansion, for a real field:
 * values[i][j] = sum_{m=-(2l-1)}^{2l-1} G^m(x_i) e^{i m phi_j}, G^{-m} = conj(G^m),
 * phi_j = 2 pi (j + 1/2)/(4l - 1) (eq. phis).  Computed as the half-sample
 * phase e^{i pi m/(4l-1)} applied to G (into the workspace) followed by one
 * complex-to-real FFT of length 4l-1 per node (cuFFT; Section 2 notes that
 * FFTs evaluate the sums over m).  G: device [2l][2l] complex (read only);
 * values: device [2l][4l-1] real.  The imaginary part of G^0 is ignored. */
sht_status sht_phi_synthesize(sht_plan_t plan, sht_precision prec, const void* G, void* values,
                              void* workspace, sht_stream_t stream);

/* Inverse of sht_phi_synthesize on band-limited data:
 * G^m(x_i) = (1/(4l-1)) sum_j values[i][j] e^{-i m phi_j}, m = 0..2l-1 (a
 * real-to-complex FFT per node, then the conjugate phase and 1/(4l-1)).
 * values: device [2l][4l-1] real (read only); G: device [2l][2l] complex. */
sht_status sht_phi_analyze(sht_plan_t plan, sht_precision prec, const void* values, void* G,
                           sht_stream_t stream);

/* Full synthesis, coefficients -> grid (Section 2, eq. expansion on the
 * tensor-product grid): the butterfly Legendre stage with the phase of eq.
 * phis fused into its unfold, writing the workspace, then the FFTs of
 * sht_phi_synthesize.  beta: device triangle; values: device [2l][4l-1]. */
sht_status sht_synthesize(sht_plan_t plan, sht_precision prec, const void* beta, void* values,
                          void* workspace, sht_stream_t stream);

/* Full analysis, grid -> coefficients: the FFTs of sht_phi_analyze into the
 * workspace, then the transposed butterfly with the conjugate phase and
 * 1/(4l-1) fused into its fold.  values: device [2l][4l-1]; beta: triangle. */
sht_status sht_analyze(sht_plan_t plan, sht_precision prec, const void* values, void* beta,
                       void* workspace, sht_stream_t stream);

/* ----------------------------------------------------------------- tracing */

/* Enables (allocating a small device buffer) or disables per-launch cycle
 * counters in the sweep kernels.  While enabled, every launch adds, summed
 * over its warps and CTAs, the clock64 cycles that warps spent executing
 * compute ops and control ops, waiting for other warps' ops (their wait
 * lists), waiting for staged values, waiting for record chunks, waiting at
 * the end-of-item barrier and publishing completions, plus the numbers of
 * compute ops, control ops and items run.  Synchronous. */
sht_status sht_trace_enable(sht_plan_t plan, int enable);

/* Copies the 16 counters (exec_gemv, exec_control, wait_dep, wait_values,
 * wait_records, wait_barrier, n_gemv, n_control, n_items, complete, 0, 0,
 * 0, 0, 0, 0) to host memory out[16]; reset != 0 zeroes them.
 * Synchronizes the device.  SHT_ERR_UNSUPPORTED if tracing is disabled. */
sht_status sht_trace_read(sht_plan_t plan, unsigned long long* out, int reset);

/* ------------------------------------------------------------ diagnostics */

/* The paper has no counterpart: measures the current device's float64
 * fused multiply-add throughput (*tflops, TFLOP/s counting 2 flops per
 * FMA) with a register-resident loop of eight independent chains per
 * thread on every SM, timed with CUDA events over one launch of about 50 ms
 * after a warm-up launch.  The ceiling the float64 kernels are compared
 * with.  Synchronous; uses the legacy default stream. */
sht_status sht_measure_fp64_fma(double* tflops);

/* The paper has no counterpart: measures the current device's float64
 * tensor-core throughput (*tflops, 2 flops per FMA) with a register-resident
 * loop of the 8x8x4 float64 warp MMA, eight independent accumulations per
 * warp on every SM, timed like sht_measure_fp64_fma.  It tells whether block
 * products over several right-hand sides could run faster on tensor cores
 * than on the FP64 FMA pipe.  Synchronous; uses the legacy default stream. */
sht_status sht_measure_fp64_mma(double* tflops);

/* ----------------------------------------------- direct float64 baseline */

/* Stores the dense operator P-bar^m_{m+p+2j}(x_{l+i}) (float64, kept rows
 * only) on the device: sum over (m,p) of rows * n_{m,p} * 8 bytes
 * (about 17.2 GB at l = 1024).  Synchronous. */
sht_status sht_direct_prepare(sht_plan_t plan);
/* Same results as the SHT_FP64 Legendre entry points, computed as dense
 * float64 products with the stored operator (the O(l^3) direct method of
 * Section 2).  Asynchronous on stream. */
sht_status sht_direct_synthesize(sht_plan_t plan, const void* beta, void* G, sht_stream_t stream);
sht_status sht_direct_analyze(sht_plan_t plan, const void* G, void* beta, sht_stream_t stream);

/* ---------------------------------------------------- one block, any size */

/* Largest bandlimit sht_unit_stats_compute accepts. */
#define SHT_UNIT_STATS_MAX_L 40000

typedef struct {
  int l, m, parity;
  int n;                 /* columns n_{m,p} */
  int rows_kept;         /* rows after trimming */
  int levels;            /* merge levels */
  int n_blocks;          /* IDs in the butterfly */
  int k_max;             /* Section 5 tables: k_max */
  double k_avg;          /* k_avg */
  double k_sigma;        /* k_sigma (population standard deviation) */
  double max_abs_T;      /* largest |entry| of an interpolation matrix */
  long long factor_values, dense_values;
  long long m_max_words; /* Section 5 tables: m_max, peak float64 words of the build */
  double t_quad, t_comp; /* seconds: nodes and weights; the depth-first build */
  double eps_fwd;        /* max |A beta (butterfly) - A beta (direct)|, beta unit-norm U(-1,1) */
  double eps_inv;        /* max |A^T mu (butterfly) - A^T mu (direct)|, mu unit-norm U(-1,1) */
  int direct;            /* 1 if the block is stored dense (compression did not pay) */
} sht_unit_stats;

/* Builds, on the host only, the butterfly of the single parity block
 * A^{m,parity}_{ij} = sqrt(2 w_{l+i}) P-bar^m_{m+parity+2j}(x_{l+i}) (the
 * weighted Gauss-Legendre block of a plan with bandlimit l, Section 4) with
 * threshold eps_id and the leaf width, trimming and band options of opts
 * (NULL: defaults), 1 <= l <= SHT_UNIT_STATS_MAX_L.  Fills *out with the
 * rank statistics and precomputation costs the paper tabulates (Section 5,
 * e.g. Table small_time / small_pre; at m = 0, parity 0 the block is the
 * matrix of the paper's even-degree transform with n = l) and the max-abs
 * errors of the butterfly and of its transpose against the direct products
 * on unit-norm vectors with entries uniform in (-1, 1) (seeded SplitMix64).
 * No CUDA calls; allocates host memory only for the duration of the call. */
sht_status sht_unit_stats_compute(int l, int m, int parity, double eps_id, const sht_plan_opts* opts,
                                  unsigned long long seed, sht_unit_stats* out);

/* The paper's own quadrature (Section 4, Lemmas zeros and quadratures): the
 * n positive zeros x[0..n) (ascending) of P-bar^m_{m+parity+2n} and their
 * weights rho[0..n) (for parity 1 the sigma_j of eq. weights2), such that
 * sqrt(rho_i) P-bar^m_{m+parity+2j}(x_i), i, j < n, is orthogonal.
 * Computed as the eigenvalues in x^2 of the Jacobi matrix of the x^2
 * recurrence (eqs. c_rec, d_rec, recurrence0, recurrence) by Sturm-sequence
 * bisection, refined by Newton steps on the recurrence; the weights from
 * the orthonormality of the rows.  Host only; x and rho are host arrays of
 * n doubles (1 <= n <= SHT_UNIT_STATS_MAX_L). */
sht_status sht_gauss_jacobi_nodes(int m, int parity, int n, double* x, double* rho);

/* As sht_unit_stats_compute, for the paper's n x n matrix of eq. transform
 * (parity 0: sqrt(rho_i) P-bar^m_{m+2j}(x_i)) or eq. transform2 (parity 1:
 * sqrt(sigma_i) P-bar^m_{m+2j+1}(y_i)) at the nodes of
 * sht_gauss_jacobi_nodes: the matrices of the paper's Tables evens and odds
 * (m = n) and small (m = 0).  t_quad is the time for those nodes and
 * weights. */
sht_status sht_unit_stats_gauss_jacobi(int n, int m, int parity, double eps_id, const sht_plan_opts* opts,
                                       unsigned long long seed, sht_unit_stats* out);

/* ------------------------------------------- the paper's matrices on the GPU */

/* Largest size of a single-block plan. */
#define SHT_GJ_MAX_N 40000

/* A plan for the paper's own n x n matrix of order m (Section 4):
 *   parity 0, eq. transform:  A[i][j] = sqrt(rho_i)   P-bar^m_{m+2j}(x_i),
 *   parity 1, eq. transform2: A[i][j] = sqrt(sigma_i) P-bar^m_{m+2j+1}(y_i),
 * i, j < n, at the nodes and weights of sht_gauss_jacobi_nodes (Lemma zeros,
 * Lemma quadratures).  The block is factored into the butterfly of Section
 * 2.2 on the host (depth-first, Section 3; eps_id as for sht_plan_create_ex)
 * and applied on the GPU level by level: each butterfly level is one launch
 * of the sweep kernel whose work items (groups of that level's blocks) spread
 * over the GPU, the vectors between levels in global memory owned by the
 * plan.  Options as sht_plan_create_ex (opts may be NULL) except that
 * device_build, plan_cache and debug_unmet_dependency must be 0 / NULL; 1 <=
 * n <= SHT_GJ_MAX_N, 0 <= m <= SHT_GJ_MAX_N.  Destroy with sht_plan_destroy;
 * sht_prepare, sht_plan_get_stats, sht_plan_stream, sht_trace_enable and
 * sht_last_device_status apply.  The order-based entry points (Legendre
 * stage, phi stage, direct baseline, batches, sht_plan_nodes, sht_plan_save)
 * refuse such a plan with SHT_ERR_UNSUPPORTED.  Returns SHT_ERR_INVALID_ARG
 * also when a butterfly level is wider than 2^20 elements. */
sht_status sht_gj_plan_create(int n, int m, int parity, double eps_id, const sht_plan_opts* opts, sht_plan_t* out);

/* The forward transform alpha = A beta (eqs. transform / transform2) and the
 * inverse transform beta = A^T alpha (A is orthogonal, Lemma quadratures).
 * beta and alpha are DEVICE arrays of n complex numbers (complex128 for
 * SHT_FP64, SHT_SPLIT32 and SHT_SPLIT32_ACC64, 16-byte aligned; complex64
 * for SHT_FP32, 8-byte aligned): the real and imaginary parts are two real
 * vectors transformed together (a real vector: imaginary parts 0).  The
 * input and output may be the same array.  Asynchronous on `stream`, one
 * launch per butterfly level (sht_gj_launches); a bounded wait that gives
 * up is reported by sht_last_device_status.  Calls on one plan must not
 * overlap on the GPU (they share the plan's vectors and work counters). */
sht_status sht_gj_forward(sht_plan_t plan, sht_precision prec, const void* beta, void* alpha, sht_stream_t stream);
sht_status sht_gj_inverse(sht_plan_t plan, sht_precision prec, const void* alpha, void* beta, sht_stream_t stream);

/* Launches one call of sht_gj_forward (direction 0) or sht_gj_inverse
 * (direction 1) makes in precision prec (building that precision's streams
 * on the host if needed). */
sht_status sht_gj_launches(sht_plan_t plan, sht_precision prec, int direction, int* launches);

/* The interpolative decomposition every butterfly block is built from
 * (Section 2.1, eq. 2.1 and Remark QR_algorithm), on the host: column-pivoted
 * Householder QR of the h x w column-major matrix A (host, not modified) to
 * the rank k at which every remaining column norm is <= eps, followed by the
 * strong rank-revealing exchanges that bound every interpolation
 * coefficient by 2 in magnitude.  Outputs (host arrays owned by the caller):
 * *k; perm[w], the k skeleton columns then the w - k others in ascending
 * order; T[k * (w - k)] (at most w^2 / 4 entries), column s holding the
 * coefficients with A[:, perm[k + s]] ~= sum_t T[s * k + t] A[:, perm[t]];
 * *swaps (if not NULL), the exchanges made.  1 <= h, 1 <= w <= 65535,
 * eps > 0. */
sht_status sht_interp_decomp(const double* A, int h, int w, double eps, int* k, int* perm, double* T, int* swaps);

/* ------------------------------------------------------------ many fields */

/* The paper transforms one function at a time.  A batch runs the Legendre
 * stage of many fields, each with its own plan (so its own bandlimit l), in
 * one persistent launch: the work items of all fields' factor streams form
 * one queue in decreasing size, so small and large fields share the GPU. */
typedef struct sht_batch_s* sht_batch_t;

#define SHT_BATCH_MAX_FIELDS 65535

/* Builds a batch of nfields fields; field f uses plans[f] (a plan may appear
 * any number of times).  Every plan must be a device plan on the same GPU
 * with the same page_bytes and consumer_warps; precision prec is built and uploaded for each
 * plan if it is not yet (as sht_prepare).  Allocates the batch's item table
 * and field table on the device.  The plans must outlive the batch. */
sht_status sht_batch_create(int nfields, const sht_plan_t* plans, sht_precision prec, sht_batch_t* out);

/* Frees the batch (NULL-safe); its plans are untouched. */
sht_status sht_batch_destroy(sht_batch_t batch);

/* Legendre synthesis of every field: for each f, the same result as
 * sht_legendre_synthesize(plans[f], prec, beta[f], G[f]).  beta and G are
 * DEVICE arrays of nfields device pointers (caller-owned, read by the
 * kernel; each entry 16-byte aligned, 8-byte for SHT_FP32).  The host checks
 * the arrays themselves; a NULL or misaligned entry is caught on the device
 * before any of that field's work starts and reported by
 * sht_batch_last_device_status as SHT_ERR_INVALID_ARG.  One launch,
 * asynchronous on stream; allocates and copies nothing, so it can be
 * captured in a CUDA graph.  Calls on one batch must not overlap in time
 * (they share its work-queue counter). */
sht_status sht_batch_synthesize(sht_batch_t batch, const void* const* beta, void* const* G, sht_stream_t stream);

/* Legendre analysis of every field (as sht_legendre_analyze per field);
 * G and beta as in sht_batch_synthesize. */
sht_status sht_batch_analyze(sht_batch_t batch, const void* const* G, void* const* beta, sht_stream_t stream);

/* Adjoint of the Legendre synthesis of every field (as
 * sht_legendre_synthesize_adjoint per field): the transposed butterfly
 * without quadrature weights, the backward pass of a loss on G.  G and beta
 * as in sht_batch_synthesize. */
sht_status sht_batch_synthesize_adjoint(sht_batch_t batch, const void* const* G, void* const* beta,
                                        sht_stream_t stream);

/* Full synthesis of every field, coefficients -> grid: for each f the same
 * values as sht_synthesize(plans[f], prec, beta[f], values[f],
 * workspace[f]).  One launch runs every field's Legendre stage with the
 * phase of eq. phis fused, writing workspace[f] (sht_workspace_bytes of plan
 * f); then each field's complex-to-real FFTs run on stream.  beta, values and
 * workspace are HOST arrays of nfields device pointers (read during the call;
 * beta and workspace entries 16-byte aligned, 8-byte for SHT_FP32).  The
 * pointer tables reach the device through a ring of four slots in stream
 * order: a call may wait on the host for the launch made four calls earlier
 * on this batch.  Not for stream capture (use sht_batch_synthesize and
 * sht_phi_synthesize per field there).  Asynchronous otherwise. */
sht_status sht_batch_synthesize_grid(sht_batch_t batch, const void* const* beta, void* const* values,
                                     void* const* workspace, sht_stream_t stream);

/* Full analysis of every field, grid -> coefficients (as sht_analyze per
 * field): each field's real-to-complex FFTs into workspace[f], then one
 * launch of every field's transposed butterfly with the conjugate phase and
 * 1/(4l-1) fused into its fold.  Arrays and ordering as in
 * sht_batch_synthesize_grid. */
sht_status sht_batch_analyze_grid(sht_batch_t batch, const void* const* values, void* const* beta,
                                  void* const* workspace, sht_stream_t stream);

/* Device status word of the batch's launches (synchronizes stream): SHT_OK,
 * SHT_ERR_TIMEOUT (a bounded wait gave up) or SHT_ERR_INVALID_ARG (a field's
 * pointer entry was NULL or misaligned).  A non-OK status is cleared. */
sht_status sht_batch_last_device_status(sht_batch_t batch, sht_stream_t stream);

/* Times the launch shapes the batch's streams allow over reps launches of
 * the given direction with these DEVICE pointer arrays, and keeps the
 * fastest for that direction.  The plans' work items are scheduled for their
 * consumer warps, which fixes the warps and the shared-memory layout of a
 * launch; what is chosen is how many fields that share a plan are applied
 * together (at most 1, 2 or 4 per group, as far as their vectors fit in
 * shared memory).  Directions: 0 synthesis, 1 analysis, 2 adjoint of
 * synthesis, 3 and 4 the Legendre launches of sht_batch_synthesize_grid
 * (beta -> workspace) and sht_batch_analyze_grid (workspace -> beta).  Runs
 * the transform (writes the outputs); synchronous. */
sht_status sht_batch_autotune(sht_batch_t batch, int direction, const void* const* in, void* const* out, int reps,
                              sht_stream_t stream);

/* Launch shape in use for a direction (any output pointer may be NULL). */
sht_status sht_batch_get_config(sht_batch_t batch, int direction, int* consumer_warps, int* nstages,
                                int* ctas_per_sm, int* smem_bytes);

/* The batched spellings of the full transform (one call per batch of
 * fields, no batch object kept by the caller).  Each call builds a batch of
 * plans[0..nfields) (as sht_batch_create), runs it through one persistent
 * launch of every field's Legendre stage plus each field's FFTs (as
 * sht_batch_synthesize_grid / sht_batch_analyze_grid), waits for stream and
 * frees the batch: SYNCHRONOUS on stream, and it allocates (the batch's
 * tables).  Repeated calls on the same plans should create one sht_batch_t
 * instead.  beta and values are HOST arrays of nfields device pointers (the
 * layouts of sht_synthesize / sht_analyze per field); workspace is one
 * caller-owned device buffer of sht_batched_workspace_bytes(nfields, plans,
 * prec) bytes, field f using the part that starts at the sum of the
 * preceding fields' sht_workspace_bytes, each rounded up to 256 bytes.
 * Errors as sht_batch_create and the grid entry points. */
size_t sht_batched_workspace_bytes(int nfields, const sht_plan_t* plans, sht_precision prec);
sht_status sht_synthesize_batched(int nfields, const sht_plan_t* plans, sht_precision prec,
                                  const void* const* beta, void* const* values, void* workspace,
                                  sht_stream_t stream);
sht_status sht_analyze_batched(int nfields, const sht_plan_t* plans, sht_precision prec,
                               const void* const* values, void* const* beta, void* workspace,
                               sht_stream_t stream);

/* Field groups of a direction (0..4 as in sht_batch_autotune): fields of a
 * batch that share a plan are applied together, each op's values staged
 * once for the whole group (as many fields per group as fit one CTA's shared
 * vectors, at most 4; sht_batch_autotune may lower the cap).  Receives the
 * largest group size class in use (1, 2 or 4) and the number of groups. */
sht_status sht_batch_get_groups(sht_batch_t batch, int direction, int* max_fields_per_group, int* groups);

/* ------------------------------------------------------ allocation-free call */

/* Static scratch slots of sht_legendre_synthesize_noalloc (32 bytes each). */
#define SHT_NOALLOC_MAX_SLOTS 32

/* The paper has no counterpart: this is a calling convention for callers
 * that may not allocate device memory on their compute path.  Computes the
 * same G as sht_legendre_synthesize (same kernel, same factor streams, same
 * layouts: beta device triangle, G device [2l][2l]) but allocates nothing,
 * builds nothing and uploads nothing.  The sweep's scratch (its work-queue
 * counter and status word) is slot `slot` of a fixed device array of
 * SHT_NOALLOC_MAX_SLOTS slots (one array per device) instead of memory the
 * plan allocated.
 *   slot:   0 <= slot < SHT_NOALLOC_MAX_SLOTS, else SHT_ERR_INVALID_ARG
 *           (sht_last_error_detail names the limit).
 *   status: optional caller-owned device word.  It is zeroed in stream
 *           order, then receives SHT_ERR_TIMEOUT if a bounded wait of the
 *           launch gave up (0 otherwise).  With NULL the launch reports into
 *           a private word of the slot that nothing reads, so a timeout
 *           cannot be detected (G is then undefined): pass a word wherever
 *           that matters.
 * The precision must already be on the device (SHT_FP64 is uploaded by
 * sht_plan_create; others by sht_prepare); otherwise SHT_ERR_UNSUPPORTED.
 * The first call on a device does a one-time set-up: it looks up the
 * array's address with the device current.  That step is not stream
 * ordered, so make the first call before any stream capture.  Calls whose
 * launches overlap in time (other streams, threads or plans) must use
 * different slots: two launches on one slot race on its counter.
 * The caller's current device is the same after the call as before it, and
 * a CUDA error the caller left pending on this thread is left pending.
 * Asynchronous on stream. */
sht_status sht_legendre_synthesize_noalloc(sht_plan_t plan, sht_precision prec, const void* beta, void* G,
                                           int slot, unsigned* status, sht_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SHT_H */
