/*
 * qtam.h -- C ABI of the GB300-native QTAM library (invertible Q-transform,
 * "Q-Transform Amplitude Modulation", arXiv 2603.29785).
 *
 * The library computes, on one GPU, the QTAM analysis (forward) and
 * canonical dual-frame synthesis (inverse) of real segments:
 *
 *   forward  (Sec. III; App. A):  X = rfft_N(x);  for every Q-plane p and
 *            log-spaced row k, S'_k[d] = W_k[k_c+d] X[k_c+d] on |d| <= h_k,
 *            shifted to baseband, zero-padded to M and inverse-transformed:
 *            Y_k[n] = (M N)^(-1/2) sum_j S'_k[j] exp(+2 pi i j n / M).
 *   inverse  (Eq. qtam_canonical_inverse; App. C):  per row the FFT of Y_k,
 *            re-scaled by sqrt(N/M) and shifted back to k_c, weighted by
 *            W_k and summed into A[f]; X_hat = A / P on the kept bins
 *            F_tau = {P > 0, P >= tau max P}, 0 elsewhere; x_hat = irfft_N.
 *
 *   W_k[f] = c_k (1 - ((f - k_c)/h_k)^2)^2 on |f - k_c| <= h_k, 0 <= f <= N/2
 *            (Eq. gwpy_window_formula, Eq. support); the App. A alternatives
 *            (Hann, Kaiser, Tukey, Planck-taper) per plan or per plane
 *   P[f]   = sum over the selected planes and rows of W_k[f]^2 (App. C frame
 *            operator), computed in FP64 on the host when the plan is made.
 *
 * Beyond the transform pair: per-plane energy / peak for optimal-plane
 * selection, uneven batches, a host round trip with overlapped copies,
 * overlap-save streaming over continuous signals, a dense (undemodulated,
 * stopband-floored) mode with a single-tile inverse, and the short DFT on
 * the tensor cores (tcgen05) for M = 8192.
 *
 * Conventions for every entry point:
 *  - Pointers named x, y, workspace are DEVICE pointers on the plan's device,
 *    owned by the caller; the library never frees them.  *_host pointers are
 *    host memory (pinned for asynchronous copies).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every launch is asynchronous on that stream; nothing
 *    synchronises unless stated.
 *  - Argument and size errors are returned synchronously before any launch.
 *    Launch errors are returned as QTAM_ERR_CUDA; asynchronous faults surface
 *    at the caller's next synchronisation.  qtam_last_error() gives a message
 *    for the calling thread's last failure.  No exception crosses the ABI.
 *  - Plans are immutable after creation except for a cache of per-mask
 *    normalisers (guarded by a mutex) and may be used from several streams at
 *    once, each call with its own workspace.
 *
 * Layouts (row-major, no padding):
 *   x      [batch][N]          real, float (compute F32) or double (F64)
 *   y      [batch][P][K][M]    complex, interleaved (re, im): float2,
 *                              bf16x2 or half2 (envelope dtype), or double2
 *   column n of a row is time n*T/M from the segment start (circular).
 */
#ifndef QTAM_H
#define QTAM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define QTAM_API __attribute__((visibility("default")))
#else
#define QTAM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qtam_plan_s* qtam_plan_t;

typedef enum {
  QTAM_OK = 0,
  QTAM_ERR_INVALID_ARG = 1,      /* null pointer, negative size, bad enum, bad mask */
  QTAM_ERR_UNSUPPORTED_SIZE = 2, /* N or M outside what the kernels handle */
  QTAM_ERR_ALIASING = 3,         /* requested n_out shorter than the largest window */
  QTAM_ERR_NO_COVERAGE = 4,      /* the selected planes cover no frequency bin */
  QTAM_ERR_OUT_OF_MEMORY = 5,    /* plan tables could not be allocated */
  QTAM_ERR_CUDA = 6,             /* a CUDA runtime call or launch failed */
  QTAM_ERR_TIMEOUT = 7,          /* a bounded device-side wait expired */
  QTAM_ERR_NO_DEVICE = 8,        /* the plan was made host-only (device = -1) */
  QTAM_ERR_WORKSPACE = 9         /* workspace smaller than qtam_workspace_size() */
} qtam_status;

/* spectral windows of App. A on |d| <= h, u = d/h: bisquare (1-u^2)^2;
 * Hann (1+cos(pi u))/2; Kaiser I0(beta sqrt(1-u^2))/I0(beta) (window_param =
 * beta); Tukey with taper fraction a (window_param = a); Planck-taper with
 * taper fraction a (window_param = a, standard continuous form). */
enum { QTAM_WIN_BISQUARE = 0, QTAM_WIN_HANN = 1, QTAM_WIN_KAISER = 2, QTAM_WIN_TUKEY = 3, QTAM_WIN_PLANCK = 4 };
/* window normalisation c_k: L2 = (sum W'^2)^(-1/2) (unit-energy window);
 * PAPER = 1 / sum W'^2 (Eq. gwpy_window_and_normalization read literally);
 * NONE = 1. */
enum { QTAM_NORM_L2 = 0, QTAM_NORM_PAPER = 1, QTAM_NORM_NONE = 2 };
enum { QTAM_DTYPE_F32 = 0, QTAM_DTYPE_F64 = 1, QTAM_DTYPE_BF16 = 2, QTAM_DTYPE_F16 = 3 };
enum { QTAM_SHORT_DFT_CUDA = 0, QTAM_SHORT_DFT_TENSOR = 1, QTAM_SHORT_DFT_AUTO = 2 };

typedef struct {
  double sample_rate;     /* f_s in Hz, > 0 */
  int64_t length;         /* N samples per segment; even, N/2 a multiple of 16 with factors 2,3,5 */
  const double* q;        /* n_q quality factors, one Q-plane each (copied) */
  int32_t n_q;            /* 1 .. 64 */
  double f_min, f_max;    /* log grid f_k = f_min (f_max/f_min)^(k/(K-1)), endpoints included */
  int32_t rows_per_plane; /* K >= 1 */
  int32_t window;         /* QTAM_WIN_*; non-bisquare windows read a per-plan W' table (compile-time
                             row variants with F32 envelopes, else the runtime engine) */
  int32_t norm;           /* QTAM_NORM_* */
  double q_width;         /* half-width h = floor(f T q_width / Q); <= 0 selects sqrt(11) */
  double max_window_hz;   /* 0: automatic clamp from the largest centre gap (App. A); > 0: manual */
  int32_t n_out;          /* M; 0: smallest 2^a 3^b 5^c >= the largest window */
  int32_t compute_dtype;  /* QTAM_DTYPE_F32 or QTAM_DTYPE_F64 */
  int32_t envelope_dtype; /* F32/BF16/F16 with F32 compute; F64 with F64 compute */
  double p_floor_rel;     /* tau; < 0 selects the default (1e-6 for F32, 0 for F64) */
  double window_param;    /* Kaiser beta in [0, 100]; Tukey / Planck taper fraction in [0, 1];
                             ignored for bisquare and Hann; anything else -> QTAM_ERR_INVALID_ARG */
  /* composite bank (App. A: planes scan Q x window x shape parameter): when
   * non-NULL, n_q entries giving plane p's window / parameter, overriding
   * `window` / `window_param` (same rules per entry).  Read during qtam_plan
   * only; the caller keeps ownership.  Planes may repeat a Q value. */
  const int32_t* plane_window;
  const double* plane_window_param;
  /* short DFT engine of the envelope stage: QTAM_SHORT_DFT_CUDA (default:
   * FP32 mixed-radix FFTs on the CUDA cores) or QTAM_SHORT_DFT_TENSOR (the
   * length-8192 DFT as a 64 x 128 four-step whose two DFT stages are BF16
   * matrix products on the tensor cores with FP32 accumulation and an FP32
   * twiddle between them; needs n_out = 8192 and F32 compute, else
   * QTAM_ERR_UNSUPPORTED_SIZE).  The inverse runs the mirrored four-step
   * (DFT-128 then twiddle then DFT-64, on the tensor cores) when the
   * envelope pointer is 16-byte aligned, else the CUDA-core rows.  Both
   * directions carry BF16 operand rounding (relative error ~3e-3).
   * QTAM_SHORT_DFT_AUTO picks the engine per plan: the tensor cores where
   * their rounding is within the plan's own accuracy class (n_out = 8192,
   * F32 compute, BF16 envelopes, no dense mode: there they are also the
   * faster engine), the CUDA cores everywhere else; qtam_plan_info reports
   * the choice. */
  int32_t short_dft;
  /* dense mode (the alternative inversion of Sec. III, beside the
   * demodulated default): stopband_eps > 0 gives every window the floor eps wherever it
   * vanishes (outside the support and at its edge points), so each tile
   * spans all N/2+1 bins; n_out (M) must then be >= N/2+1 (default: the
   * smallest 2^a 3^b 5^c above it) and any single tile inverts by spectral
   * division (qtam_inverse_single_tile).  remodulate = 1 multiplies the
   * envelopes by exp(+2 pi i k_c n / M): the undemodulated tile, i.e. the
   * inverse DFT of the unshifted filtered spectrum X W_k.  Both run on the
   * CUDA cores: the compile-time row variants built for the dense mode
   * where the length has them (FP32 compute, any envelope storage;
   * M = 4320), else
   * the runtime engine, which also serves the single-tile inverse;
   * remodulate combined with short_dft = TENSOR, or eps with it, is
   * QTAM_ERR_UNSUPPORTED_SIZE. */
  double stopband_eps;
  int32_t remodulate;
} qtam_plan_desc;

typedef struct {
  int64_t length;                 /* N */
  int64_t n_bins;                 /* N/2 + 1 */
  int32_t n_planes;               /* P */
  int32_t rows_per_plane;         /* K */
  int32_t n_out;                  /* M */
  int32_t h_max;                  /* clamp half-width (huge when unclamped) */
  int32_t max_window;             /* max_k L_k = 2 h_k + 1 */
  int32_t compute_dtype;
  int32_t envelope_dtype;
  int32_t fft_n1, fft_n2;         /* four-step split of the N/2-point long FFT */
  int64_t envelope_bytes_per_segment; /* P*K*M * bytes per complex */
  int64_t band_bins;              /* sum over rows of the in-band window bins */
  double p_floor_rel;             /* tau in use */
  double kappa;                   /* max over kept bins of max_k W_k / P (all planes) */
  int64_t kept_bins;              /* |F_tau| for all planes */
  int64_t device_bytes;           /* bytes of resident plan tables on the device */
  int32_t row_variant;            /* CUDA-core row-kernel variant in use (-1: runtime engine); with
                                     the tensor-core short DFT it serves only an inverse of
                                     envelopes that are not 16-byte aligned */
  int32_t short_dft;              /* QTAM_SHORT_DFT_* engine of the envelope stage */
  double stopband_eps;            /* dense mode floor (0: off) */
  int32_t remodulate;             /* 1: envelopes carry the carrier exp(+2 pi i k_c n / M) */
} qtam_plan_info_t;

/* Fill *d with defaults: bisquare, L2 norm, q_width sqrt(11), automatic clamp
 * and n_out, F32 compute and envelopes, default floor.  Sizes stay zero. */
QTAM_API void qtam_plan_desc_init(qtam_plan_desc* d);

/* Build a plan (App. A geometry, FP64 frame operator, twiddle tables) and
 * upload its tables to `device`.  device = -1 makes a host-only plan whose
 * geometry can be queried but which cannot run transforms.  The plan owns its
 * device tables until qtam_destroy.  Synchronous. */
QTAM_API qtam_status qtam_plan(const qtam_plan_desc* desc, int device, qtam_plan_t* out);

QTAM_API qtam_status qtam_plan_info(qtam_plan_t plan, qtam_plan_info_t* out);

/* Per-row geometry, row r = p*K + k, each array caller-owned with P*K
 * entries (any may be NULL): centre frequency f_k (Hz), centre bin k_c,
 * half-width h_k and normalisation c_k. */
QTAM_API qtam_status qtam_plan_rows(qtam_plan_t plan, double* f, int64_t* kc, int32_t* h, double* c);

/* Frame operator P[f], f = 0..N/2, of the planes in plane_mask (bit p =
 * plane p; 0 = all planes), FP64, into the caller's host array of N/2+1. */
QTAM_API qtam_status qtam_frame_operator(qtam_plan_t plan, uint64_t plane_mask, double* p_out);

/* Row-kernel variants (launch shapes) usable for this plan: the runtime
 * mixed-radix engine (-1, any length) and the compile-time variants built for
 * the plan's envelope length M (FP32 compute).  Writes up to `capacity` ids
 * into `ids` and the total into *count.  All variants compute the same
 * transform; they differ in radix sequence, rows per block and occupancy.
 * An autotuner times them (qtam_stage_envelopes / qtam_stage_accumulate)
 * and keeps the fastest with qtam_plan_set_variant. */
QTAM_API qtam_status qtam_plan_variants(qtam_plan_t plan, int32_t* ids, int32_t capacity, int32_t* count);

/* Select the row-kernel variant for subsequent calls on this plan.  Not
 * synchronised with calls running concurrently on other threads. */
QTAM_API qtam_status qtam_plan_set_variant(qtam_plan_t plan, int32_t variant);

/* Describe a variant: a name (radices, rows per block, occupancy target)
 * into name[capacity], threads per block and rows per block. */
QTAM_API qtam_status qtam_variant_describe(int32_t variant, char* name, size_t capacity, int32_t* threads,
                                           int32_t* rows_per_block);

/* Bytes of device workspace one qtam_forward/qtam_inverse call on `batch`
 * segments needs (the long-FFT buffers and the spectrum accumulator). */
QTAM_API qtam_status qtam_workspace_size(qtam_plan_t plan, int64_t batch, size_t* bytes);

/* QTAM analysis of `batch` segments: x [batch][N] -> y [batch][P][K][M].
 * batch = 0 is a no-op.  workspace_bytes must be >= qtam_workspace_size. */
QTAM_API qtam_status qtam_forward(qtam_plan_t plan, const void* x, int64_t batch, void* y,
                         void* workspace, size_t workspace_bytes, void* stream);

/* QTAM synthesis by the canonical dual frame of the planes in plane_mask
 * (0 = all): y [batch][P][K][M] -> x [batch][N].  Rows of unselected planes
 * are not read.  Any y is accepted (e.g. masked or row-zeroed envelopes). */
QTAM_API qtam_status qtam_inverse(qtam_plan_t plan, const void* y, int64_t batch, uint64_t plane_mask,
                         void* x, void* workspace, size_t workspace_bytes, void* stream);

/* Stage entry points of the same path, for stage-level checks and custom
 * pipelines.  spectrum: x -> X [batch][N/2+1] complex (step a1).
 * envelopes: X -> y (steps a2-a4).  accumulate: y -> A [batch][N/2+1]
 * complex, zeroed first (steps a5-a6).  synthesize: A -> x with the 1/P of
 * plane_mask and the inverse long FFT (step a7).  workspace as above. */
QTAM_API qtam_status qtam_stage_spectrum(qtam_plan_t plan, const void* x, int64_t batch, void* X,
                                void* workspace, size_t workspace_bytes, void* stream);
QTAM_API qtam_status qtam_stage_envelopes(qtam_plan_t plan, const void* X, int64_t batch, void* y, void* stream);
QTAM_API qtam_status qtam_stage_accumulate(qtam_plan_t plan, const void* y, int64_t batch, uint64_t plane_mask,
                                  void* A, void* stream);
QTAM_API qtam_status qtam_stage_synthesize(qtam_plan_t plan, const void* A, int64_t batch, uint64_t plane_mask,
                                  void* x, void* workspace, size_t workspace_bytes, void* stream);

/* Single-tile inverse of the dense mode: x[b] = irfft( T~_k / W_k ) from the
 * one tile (plane, row) of y [batch][P][K][M] -- the tile's spectrum shifted
 * back to its carrier and divided by its (floored) window on every bin.
 * Needs stopband_eps > 0 (else QTAM_ERR_INVALID_ARG); other tiles are not
 * read.  Workspace as for qtam_inverse. */
QTAM_API qtam_status qtam_inverse_single_tile(qtam_plan_t plan, const void* y, int64_t batch, int32_t plane,
                                              int32_t row, void* x, void* workspace, size_t workspace_bytes,
                                              void* stream);

/* Forward then inverse from HOST buffers: copies x_host into x_dev, runs
 * qtam_forward into y_dev and qtam_inverse into xhat_dev, and copies xhat_dev
 * back into xhat_host; synchronises `stream` before returning.  The batch is
 * split into inner chunks of about 16 MB of input and short first and last
 * chunks (about batch/16 segments; at most 10 chunks): host-to-device
 * copies run on one library-owned stream and device-to-host copies on
 * another, ordered against the transforms by events, so the copies of
 * neighbouring chunks overlap the transforms (pinned host buffers make the
 * copies asynchronous).  Even chunks are transformed on `stream`; when the
 * workspace holds two workspaces of the largest chunk (and is 256-byte
 * aligned), odd chunks run on a third library-owned stream in the second
 * one, so neighbouring chunks' kernels overlap.  One round trip at a time
 * per plan (calls on the same plan serialise).  All device buffers are caller-owned
 * ([batch][N], [batch][P][K][M], [batch][N]); workspace as for qtam_forward
 * with `batch` segments. */
QTAM_API qtam_status qtam_roundtrip_host(qtam_plan_t plan, const void* x_host, int64_t batch, uint64_t plane_mask,
                                void* xhat_host, void* x_dev, void* y_dev, void* xhat_dev,
                                void* workspace, size_t workspace_bytes, void* stream);

/* Signal-quality metrics per Q-plane for optimal-plane selection (App. A,
 * multi-Q bank, "optimal selection" mode): for every segment b and plane p,
 * energy[b*P + p] = sum over rows and columns of |Y|^2 (accumulated in FP64)
 * and peak[b*P + p] = max |Y|^2.  The plane with the largest energy (or peak)
 * of each segment is its optimal plane.  energy (double) and peak (float) are
 * device arrays of batch*P entries. */
QTAM_API qtam_status qtam_plane_metrics(qtam_plan_t plan, const void* y, int64_t batch, double* energy, float* peak,
                                        void* stream);

/* Multiply every envelope row by a gain: y[b][p][k][*] *= gain[(b*P + p)*K + k]
 * (gain: device float array of batch*P*K entries).  Gain 0 zeroes a row --
 * the masked (row-zeroed) envelopes the inverse accepts; gain 1 leaves the
 * row untouched.  A pre-processing step for synthesis from a subset of the
 * tiles (cluster masks, App. C canonical dual of the kept rows). */
QTAM_API qtam_status qtam_scale_rows(qtam_plan_t plan, void* y, int64_t batch, const float* gain, void* stream);

/* One group of equal-length segments of a batched call: `batch` segments
 * transformed with `plan`.  forward reads x [batch][N] and writes y
 * [batch][P][K][M]; inverse reads y and writes x.  Pointers are device
 * buffers of the plans' device, owned by the caller. */
typedef struct {
  qtam_plan_t plan;
  const void* in;
  void* out;
  int64_t batch;
} qtam_group;

/* Workspace bytes for a batched call over these groups: the largest
 * single-group workspace (groups run in stream order and share it). */
QTAM_API qtam_status qtam_batched_workspace_size(const qtam_group* groups, int32_t n_groups, size_t* bytes);

/* Segments of uneven length (one group per plan) in one call: every group's
 * forward transform (in = x, out = y), enqueued in order on `stream`.  All
 * plans must live on the same device.  The whole call can be captured into
 * one CUDA graph (no allocation, no synchronisation inside); make one
 * uncaptured call first so plane-mask tables and kernel attributes exist. */
QTAM_API qtam_status qtam_forward_batched(const qtam_group* groups, int32_t n_groups, void* workspace,
                                          size_t workspace_bytes, void* stream);

/* Batched inverse (in = y, out = x) with the canonical dual of plane_mask. */
QTAM_API qtam_status qtam_inverse_batched(const qtam_group* groups, int32_t n_groups, uint64_t plane_mask,
                                          void* workspace, size_t workspace_bytes, void* stream);

/* qtam_forward without a workspace argument, for callers that cannot
 * allocate device memory at call time (real-time loops, host callbacks where
 * a cudaMalloc would stall, plug-ins whose host application owns all device
 * memory).  The paper has no counterpart: this is a library convenience.
 * The long-FFT scratch lives in a fixed 32 MiB array inside the library,
 * reserved on every GPU that loads it until the process exits; a batch whose
 * qtam_workspace_size exceeds 32 MiB returns QTAM_ERR_WORKSPACE.  The call
 * itself allocates nothing.  All calls on a device share that array: calls
 * whose kernels may overlap on the GPU (unordered streams) race and must be
 * serialised by the caller.  The first call on each device looks up the
 * array's address; make it before any stream capture.  A call with
 * batch == 0 on a device plan returns QTAM_OK without that lookup and
 * without launching anything. */
QTAM_API qtam_status qtam_forward_noalloc(qtam_plan_t plan, const void* x, int64_t batch, void* y, void* stream);

/* ---- Streaming analysis of a continuous signal (overlap-save) ----------
 * The paper motivates hours-long signals (Sec. I) without fixing a scheme;
 * this is overlap-save over the plan's segment length N.  Chunks of N
 * samples advance by `hop` samples; the guard G = (N - hop)/2 on each side
 * absorbs the circular wrap of each chunk's transform and only the central
 * Hn = hop*M/N envelope columns of a chunk are kept.  hop and G must be
 * multiples of the column quantum N / gcd(N, M), where column and sample
 * boundaries coincide.  A chunk starting a samples after the stream origin
 * has its envelope rows multiplied by exp(-2 pi i k_c a / N), so every chunk
 * is demodulated against the same time origin and the map is continuous
 * across chunks.  A remodulated plan's tiles already carry their carrier on
 * absolute time (a shift of the input only shifts their columns), so their
 * factor is 1.  The stream starts after 2G zero samples: map column c is
 * time c*N/M - G (forward delay G), and the streaming inverse returns sample
 * s at time s - 2G (a further G).
 *
 * The stream object keeps the last 2G input samples and the last 2G*M/N map
 * columns of every row as history, plus scratch for `max_chunks` chunks per
 * internal step (pushes longer than that run in several steps).  It owns
 * its device memory (allocated in qtam_stream_create, freed by
 * qtam_stream_destroy) and references the plan, which must outlive it.  A
 * stream's calls must be ordered on the GPU (one CUDA stream, or events). */
typedef struct qtam_stream_s* qtam_stream_t;

typedef struct {
  int64_t hop;         /* samples per chunk step */
  int64_t guard;       /* G = (N - hop) / 2 */
  int64_t quantum;     /* N / gcd(N, M) */
  int32_t hop_cols;    /* Hn = hop * M / N map columns per chunk */
  int32_t guard_cols;  /* G * M / N */
  int64_t max_chunks;  /* chunks per internal step */
  int64_t samples_in;  /* samples consumed by qtam_stream_forward since create / reset */
  int64_t columns_in;  /* map columns consumed by qtam_stream_inverse since create / reset */
  int64_t device_bytes;
} qtam_stream_info_t;

/* Create a stream over a device plan.  hop = 0 selects N/2 rounded down to
 * the quantum grid.  max_chunks >= 1.  Errors: QTAM_ERR_INVALID_ARG (hop or
 * guard off the quantum grid, hop > N), QTAM_ERR_NO_DEVICE (host-only plan),
 * QTAM_ERR_OUT_OF_MEMORY.  Synchronous. */
QTAM_API qtam_status qtam_stream_create(qtam_plan_t plan, int64_t hop, int64_t max_chunks, qtam_stream_t* out);
QTAM_API qtam_status qtam_stream_info(qtam_stream_t s, qtam_stream_info_t* out);

/* Push n samples (device, the plan's real dtype; n a multiple of hop) and
 * receive their (n/hop)*Hn map columns: y is a device array [P][K][n/hop*Hn]
 * of the plan's envelope dtype (interleaved complex), each row contiguous.
 * n = 0 is a no-op.  Enqueued on `stream`. */
QTAM_API qtam_status qtam_stream_forward(qtam_stream_t s, const void* x, int64_t n, void* y, void* stream);

/* Push n_cols map columns (device [P][K][n_cols], n_cols a multiple of Hn;
 * any values, e.g. a masked map) and receive (n_cols/Hn)*hop samples of the
 * canonical-dual reconstruction of the planes in plane_mask (0 = all). */
QTAM_API qtam_status qtam_stream_inverse(qtam_stream_t s, const void* y, int64_t n_cols, uint64_t plane_mask,
                                         void* x, void* stream);

/* Zero both histories and positions (enqueued on `stream`). */
QTAM_API qtam_status qtam_stream_reset(qtam_stream_t s, void* stream);

/* Free the stream's device memory (synchronises the device first).  NULL is a no-op. */
QTAM_API qtam_status qtam_stream_destroy(qtam_stream_t s);

/* ---- Tensor-core building block check ------------------------------------
 * One 128 x N x K BF16 matrix product on the fifth-generation tensor cores
 * (tcgen05: shared-memory operands, FP32 accumulator in tensor memory), the
 * building block of the tensor-core short DFT: D[128][N] = A[128][K] *
 * B[N][K]^T with A, B row-major BF16 (raw 16-bit patterns) and D row-major
 * FP32, all device buffers owned by the caller; flags bit 0 negates A, bit 1
 * negates B, bit 2 stages A in the M-major shared-memory layout, bit 3
 * issues no MMA so the bounded completion wait runs out after about 1 ms
 * (the timeout path: counted by qtam_tc_status, tensor memory released, D
 * left untouched, the context stays usable).  N, K multiples of 16 in [16, 256]; A, B 16-byte aligned.
 * Enqueued on `stream`; a tensor-core wait that runs out (about 1 s) is
 * counted and reported by qtam_tc_status. */
QTAM_API qtam_status qtam_tc_gemm_check(const void* A, const void* B, float* D, int32_t N, int32_t K, int32_t flags,
                                        void* stream);
/* Number of bounded tensor-core waits that ran out since the library was
 * loaded on the current device (0 when every tensor-core kernel completed).
 * Synchronous. */
QTAM_API qtam_status qtam_tc_status(int32_t* timeouts);

/* Release the plan's device tables and the plan.  NULL is a no-op. */
QTAM_API qtam_status qtam_destroy(qtam_plan_t plan);

QTAM_API const char* qtam_status_string(qtam_status s);
QTAM_API const char* qtam_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* QTAM_H */
