/*
 * uwb.h -- C ABI of the GB300 segment-search confocal imaging library.
 *
 * Method: Ettefagh, Moghaddam, Vahidian, "A Novel Low-Complexity Framework in
 * Ultra-Wideband Imaging for Breast Cancer Detection" (arXiv:1709.02549):
 * monostatic confocal DAS (Section II.A, Eq. 1 and Eq. 3) and DMAS
 * (Section II.B) images, evaluated only where the coarse-to-fine segment
 * search of Section III asks for them (spatial decimation, ROI selection with
 * the Eq. 5 metric and the Eq. 6-7 stopping rule, sliding framing, final
 * full-resolution imaging of the ROI).
 *
 * Conventions shared by every entry point
 *  - Every array argument is a DEVICE pointer owned by the caller; the library
 *    never frees or keeps it. uwb_grid and uwb_rule are HOST structs, read
 *    during the call only.
 *  - traces: float32, [batch][M][N] row-major (scan, antenna, sample); sample n
 *    of antenna i is the echo at time n / fs. Samples outside [0, N) read as 0.
 *  - antennas: float32 [M][3] metres (x, y, z), shared by every scan when
 *    antenna_stride == 0, else scan b uses antennas + b * antenna_stride.
 *  - Focal grid: point (ix, iy, iz) sits at origin + (ix, iy, iz) * pitch;
 *    images are [batch][nz][ny][nx] float32 with x fastest. 2-D grids have
 *    dim == 2 and n[2] == 1.
 *  - Delay: round trip tau_i(r) = 2 |r - a_i| / v, in samples u_i = tau_i fs
 *    (Eq. 1, read with the round trip and the medium speed v; the printed
 *    form divides by 2 and uses c). The aligned signal is
 *    x_i(k) = Y_i(u_i - floor(W/2) + k), k = 0..W-1, linearly interpolated.
 *  - DAS energy  I(r) = sum_k (sum_i x_i(k))^2                      (Eq. 3)
 *    DMAS energy I(r) = sum_k (sum_{i<j} x_i(k) x_j(k))^2      (Section II.B)
 *    UWB_DMAS forms the pair sum as ((sum_i x_i)^2 - sum_i x_i^2) / 2;
 *    UWB_DMAS_LITERAL multiplies every pair. Both compute the same quantity.
 *  - Arithmetic is float32 (delays, interpolation, accumulation); the segment
 *    metrics of uwb_localize are float64.
 *  - Every call is asynchronous on `stream` (a cudaStream_t passed as void*,
 *    NULL = legacy default stream) and returns a status: UWB_OK or a negative
 *    UWB_ERR_* code for errors found on the host before any launch.
 *    uwb_last_error() describes the last failure of the calling thread.
 *    Errors found on the device (a bounded wait that ran out, non-finite
 *    energies) are reported in uwb_result.status or by uwb_device_status().
 *  - Staging waits inside kernels are bounded; a kernel that gives up records
 *    UWB_ERR_TIMEOUT instead of hanging. A CTA that gives up leaves after one
 *    more bounded wait even if its copy is still in flight, and that copy may
 *    still land in shared memory another CTA of the same launch then uses:
 *    once UWB_ERR_TIMEOUT is reported, treat every output of that call as
 *    invalid, not only the scans it names. Launches that hand out tiles
 *    through a counter stop handing them out after such a timeout.
 *  - Image launches with at least 4 tiles per CTA and several CTAs per SM
 *    hand tiles out through a counter. uwb_localize, uwb_localize_batch,
 *    uwb_localize_batch_noalloc, uwb_localize_host,
 *    uwb_localize_multistatic_batch and the plan calls own their counters in
 *    their workspace and zero them themselves, so their launches split
 *    dynamically in a CUDA graph too. The other entry points take a counter
 *    from a per-device pool of 64 (reused only after the launch that used it
 *    has completed); launched under stream capture, or while every counter
 *    is busy, they split tiles into equal contiguous ranges instead. Results
 *    do not depend on the split.
 */
#ifndef UWB_H
#define UWB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define UWB_OK 0
#define UWB_ERR_ARG -1          /* invalid argument (null pointer, size, range) */
#define UWB_ERR_CUDA -2         /* a CUDA runtime / driver call failed */
#define UWB_ERR_TIMEOUT -3      /* a bounded device wait ran out */
#define UWB_ERR_NONFINITE -4    /* NaN or Inf in the decimated energy profile */
#define UWB_ERR_UNSUPPORTED -5  /* sizes outside what this build handles */
#define UWB_ERR_WORKSPACE -6    /* workspace missing, misaligned or too small */
#define UWB_ERR_BOUNDS -7       /* bounds-checked builds only (compiled with -DUWB_CHECK): an image
                                   kernel computed a staged-window, image or profile index outside
                                   its buffer; the access was redirected inside it and the call's
                                   outputs are invalid */

/* beamformers */
#define UWB_DAS 0
#define UWB_DMAS 1            /* pair sum through ((sum x)^2 - sum x^2) / 2 */
#define UWB_DMAS_LITERAL 2    /* pair sum by multiplying every pair i < j */

/* spatial decimation modes (Section III, "Spatial Decimation") */
#define UWB_DECIM_MANUAL 0    /* factor given in uwb_rule.decimation */
#define UWB_DECIM_AUTO 1      /* from uwb_rule.min_tumor_diameter (Section IV) */

/* decision metrics (Section III, "ROI Selection") */
#define UWB_METRIC_HYBRID 0            /* Eq. 5, weight clipped to [0, 1] */
#define UWB_METRIC_MEAN 1
#define UWB_METRIC_VARIANCE 2
#define UWB_METRIC_HYBRID_UNCLIPPED 3  /* Eq. 5 exactly as printed */

/* why the selection loop stopped */
#define UWB_STOP_NONE 0
#define UWB_STOP_METRIC 1     /* Eq. 6-7: between-class scatter stopped growing or
                                 within-class scatter stopped shrinking */
#define UWB_STOP_MINSIZE 2    /* no child segment was large enough to choose */
#define UWB_STOP_CAP 3        /* iteration cap reached */
#define UWB_STOP_NO_TARGET 4  /* every decimated energy is zero */
#define UWB_STOP_LEARNED 5    /* the learned proposal chose the final region */

#define UWB_MAX_ITERS 32

/* Focal-point lattice (Section II.A: the imaged region is sampled at focal
 * points spaced by the target resolution). n[0] * n[1] * n[2] must stay below
 * 2^31 - 4096 (UWB_ERR_ARG). */
typedef struct uwb_grid {
  int dim;           /* 2 or 3 */
  int n[3];          /* points per axis; n[2] == 1 when dim == 2 */
  double origin[3];  /* position of point (0,0,0) in metres */
  double pitch[3];   /* spacing per axis in metres (the final resolution) */
} uwb_grid;

/* Decision rule of the segment search (Section III). */
typedef struct uwb_rule {
  int mode;                   /* UWB_DECIM_MANUAL | UWB_DECIM_AUTO */
  int decimation;             /* manual factor D >= 1 */
  double min_tumor_diameter;  /* auto: D = floor(d / (sqrt(2) * min pitch)), >= 1 */
  int metric;                 /* UWB_METRIC_* */
  int min_segment;            /* a child segment needs every side >= this many points */
  int frame_num, frame_den;   /* sliding framing: a chosen child grows by
                                 ceil(frame_num / frame_den * side) points per side */
  int max_iters;              /* 0 = ceil(log2(max grid side)) + 2; <= UWB_MAX_ITERS */
} uwb_rule;

/* Result of one localised scan; written by the device. */
typedef struct uwb_result {
  int status;             /* UWB_OK or UWB_ERR_NONFINITE / UWB_ERR_TIMEOUT */
  int iters;              /* accepted segmentations (Table I's iteration count) */
  int n_logged;           /* iterations performed; the last may have been rejected */
  int stop_reason;        /* UWB_STOP_* */
  int decim;              /* spatial decimation factor D */
  int offset[3];          /* decimated lattice: offset per axis */
  int dcount[3];          /*                    points per axis */
  int roi_lo[3];          /* final region, full-resolution index box [lo, hi) */
  int roi_hi[3];
  int loc_idx[3];         /* argmax of the final image; -1 when there is none */
  long long points_evaluated;  /* decimated points + final-region points */
  double loc_xyz[3];      /* position of loc_idx in metres */
  double peak;            /* energy at loc_idx */
  double profile_max;     /* largest decimated energy */
  int child[UWB_MAX_ITERS];        /* chosen child per iteration: bit 0 = high x
                                      half, bit 1 = high y, bit 2 = high z */
  int n_children[UWB_MAX_ITERS];   /* candidate children per iteration */
  int box_lo[UWB_MAX_ITERS][3];    /* framed region chosen per iteration */
  int box_hi[UWB_MAX_ITERS][3];
  double metric_top[UWB_MAX_ITERS];  /* winning metric */
  double metric_gap[UWB_MAX_ITERS];  /* (top - runner-up) / |top|; 1e300 if alone */
  double between[UWB_MAX_ITERS];     /* Eq. 7 between-class scatter B_i */
  double within[UWB_MAX_ITERS];      /* Eq. 6 within-class scatter W_i */
  double stop_margin[UWB_MAX_ITERS]; /* relative margin of the continue/stop test */
} uwb_result;

/* Defaults: automatic decimation for a 1 cm tumour, hybrid metric,
 * min_segment 4, framing 1/4, default iteration cap. Returns UWB_OK or
 * UWB_ERR_ARG for a null pointer. */
int uwb_default_rule(uwb_rule* rule);

/* Spatial decimation factor D the rule gives on this grid (Section III
 * manual/automatic modes; Section IV worked example: 1 cm tumour at 1 mm
 * resolution gives 7). Returns D >= 1, or UWB_ERR_ARG. */
int uwb_decimation(const uwb_grid* grid, const uwb_rule* rule);

/* Full-resolution DAS image of one scan (Eq. 1 + Eq. 3) over every focal
 * point of `grid`. image: [nz][ny][nx] float32 output. peak_index: optional
 * ([1] int64): the linear index of the image maximum (lowest index on ties),
 * or -1 for an empty grid; NULL to skip. */
int uwb_das_image(const float* traces, int M, int N, const float* antennas,
                  const uwb_grid* grid, double v, double fs, int window,
                  float* image, long long* peak_index, void* stream);

/* Full-resolution DMAS image of one scan (Section II.B); literal_pairs != 0
 * multiplies every antenna pair, 0 uses the algebraic pair-sum identity. */
int uwb_dmas_image(const float* traces, int M, int N, const float* antennas,
                   const uwb_grid* grid, double v, double fs, int window,
                   int literal_pairs, float* image, long long* peak_index,
                   void* stream);

/* Batched full-resolution images: `batch` scans of equal M, N and grid in one
 * launch. traces [batch][M][N]; image [batch][P]; peak_index [batch] or NULL.
 * beamformer: UWB_DAS | UWB_DMAS | UWB_DMAS_LITERAL. */
int uwb_image_batch(int batch, int beamformer, const float* traces, int M, int N,
                    const float* antennas, long long antenna_stride,
                    const uwb_grid* grid, double v, double fs, int window,
                    float* image, long long* peak_index, void* stream);

/* ---- Ragged batches -----------------------------------------------------
 * Scans with different antenna counts, trace lengths, grids (same
 * dimensionality) and media, in one set of launches, with traces stored as
 * float32, float16 or bfloat16 (delays and accumulation stay float32). */
#define UWB_F32 0
#define UWB_F16 1
#define UWB_BF16 2

typedef struct uwb_scan {
  const void* traces;      /* device [M][N], element type of the plan, row-major */
  const float* antennas;   /* device [M][3] metres */
  int M, N;
  uwb_grid grid;
  double v, fs;
} uwb_scan;

typedef struct uwb_plan uwb_plan;  /* opaque host object owned by the caller */

/* Builds a plan for `batch` scans (host array, copied): per-scan descriptors,
 * tensor maps, decimated lattices (the rule applies to each scan's own grid)
 * and work offsets. Returns NULL and sets *status (if given) on error: every
 * scan must pass the checks of uwb_localize, and all share grid.dim. */
uwb_plan* uwb_plan_create(int batch, const uwb_scan* scans, int dtype, int window,
                          int beamformer, const uwb_rule* rule, int* status);
/* Device workspace the plan needs (256-byte aligned, owned by the caller). */
size_t uwb_plan_workspace(const uwb_plan* plan);
/* Element offset of scan `scan`'s image in the concatenated image array of
 * uwb_plan_images (scan == batch gives the total). -1 on error. */
long long uwb_plan_image_offset(const uwb_plan* plan, int scan);
/* Copies the plan into the workspace (queued on stream). After it, the two
 * calls below launch kernels only, so a sequence of them can be captured in
 * a CUDA graph; the workspace is reused by every run of the plan. */
int uwb_plan_upload(uwb_plan* plan, void* workspace, size_t ws_bytes, void* stream);
/* Full-resolution images of every scan (each scan's [nz][ny][nx] image at its
 * uwb_plan_image_offset) and optional per-scan argmax indices. */
int uwb_plan_images(uwb_plan* plan, float* images, long long* peak_index, void* stream);
/* The segment-search framework on every scan; out: [batch] uwb_result. */
int uwb_plan_localize(uwb_plan* plan, uwb_result* out, void* stream);
void uwb_plan_destroy(uwb_plan* plan);

/* Tile shapes of the image kernel. {0, 0, 0} = linear tiles (the default):
 * tile t of a lattice holds its points t*P .. t*P + P - 1 in x-fastest order
 * (P = 256 focal points per CTA, 128 for UWB_DMAS_LITERAL), so lattices whose
 * sides are not multiples of a tile leave no partly empty warps. Otherwise a
 * shaped tile: focal points per CTA along x, y, z, powers of two multiplying
 * to P, z = 1 for 2-D.
 * uwb_autotune runs the given batch through uwb_plan_localize once per
 * candidate shape (timed with CUDA events after a warm-up run), keeps the
 * fastest for this beamformer and dimensionality in a process-wide table
 * that later plans and uniform calls use, and reports it (tile_out, ms_out:
 * host, optional). It synchronises the stream: call it before any stream
 * capture. workspace: at least uwb_plan_workspace of a plan of the batch.
 * uwb_set_tile_shape sets the table entry (tile NULL restores the default);
 * uwb_tile_shape reads the shape currently in use. */
int uwb_autotune(int batch, const uwb_scan* scans, int dtype, int window, int beamformer,
                 const uwb_rule* rule, void* workspace, size_t ws_bytes, uwb_result* out,
                 int tile_out[3], float* ms_out, void* stream);
int uwb_set_tile_shape(int beamformer, int dim, const int tile[3]);
int uwb_tile_shape(int beamformer, int dim, int tile[3]);

/* Multistatic images (Section II.A: Eq. 2 delays; Eq. 4 DAS, DMAS over pairs
 * of channels): channel c is the echo sent by antenna channels[2c] and
 * received by antenna channels[2c+1] (int32 [C][2], device), its trace is
 * traces[b][c][0..N) and its delay in samples (|r - a_tx| + |r - a_rx|) fs / v.
 * Eq. 4 sums over every (i, j) pair; any subset may be given. antennas:
 * [M][3]. beamformer: UWB_DAS or UWB_DMAS (the literal pair form is built for
 * monostatic data only: UWB_ERR_UNSUPPORTED). A channel index outside
 * [0, M) is recorded as UWB_ERR_ARG in the device status word and clamped.
 * Otherwise as uwb_image_batch. */
int uwb_image_multistatic_batch(int batch, int beamformer, const float* traces, int C, int N,
                                const int* channels, const float* antennas, int M,
                                long long antenna_stride, const uwb_grid* grid, double v,
                                double fs, int window, float* image, long long* peak_index,
                                void* stream);

/* The segment-search framework (Section III) on multistatic scans; arguments
 * as uwb_image_multistatic_batch and uwb_localize_batch. */
size_t uwb_localize_multistatic_workspace(int batch, int C, int N, const uwb_grid* grid,
                                          int beamformer, const uwb_rule* rule);
int uwb_localize_multistatic_batch(int batch, const float* traces, int C, int N,
                                   const int* channels, const float* antennas, int M,
                                   long long antenna_stride, const uwb_grid* grid, double v,
                                   double fs, int window, int beamformer, const uwb_rule* rule,
                                   void* workspace, size_t ws_bytes, uwb_result* out,
                                   float* image, void* stream);

/* Bytes of device workspace uwb_localize_batch needs for these sizes
 * (0 on invalid arguments). The workspace must be 256-byte aligned. */
size_t uwb_localize_workspace(int batch, int M, int N, const uwb_grid* grid,
                              int beamformer, const uwb_rule* rule);

/* The segment-search framework (Section III) on one scan, entirely on the
 * device: decimated profile, normalisation to its maximum, ROI selection
 * loop (Eq. 5 metric, Eq. 6-7 stopping rule, sliding framing), final
 * full-resolution imaging of the ROI and its argmax. out: [1] uwb_result
 * (device). image: optional [P] float32; when given, the decimated energies
 * and the final-region energies are written at their focal points (the
 * paper's mixed-resolution final image) and other points are left untouched.
 * workspace: device memory of at least uwb_localize_workspace(1, ...) bytes,
 * owned by the caller, not kept after the stream reaches the end of the call. */
int uwb_localize(const float* traces, int M, int N, const float* antennas,
                 const uwb_grid* grid, double v, double fs, int window,
                 int beamformer, const uwb_rule* rule, void* workspace,
                 size_t ws_bytes, uwb_result* out, float* image, void* stream);

/* uwb_localize over `batch` independent scans in one set of launches. Scans
 * share M, N, grid, v, fs, window and rule. out: [batch]; image [batch][P]
 * or NULL. */
int uwb_localize_batch(int batch, const float* traces, int M, int N,
                       const float* antennas, long long antenna_stride,
                       const uwb_grid* grid, double v, double fs, int window,
                       int beamformer, const uwb_rule* rule, void* workspace,
                       size_t ws_bytes, uwb_result* out, float* image, void* stream);

/* Tumour-presence test (Section IV, last paragraph): localise every scan
 * twice, with the rule's decimation factor and with the manual factor
 * `decimation2`; a scan whose two runs locate the same focal point has its
 * tumour confirmed (present[b] = 1), otherwise it is declared tumour-free
 * (present[b] = 0, also when a run located nothing or failed). out1, out2:
 * [batch] uwb_result (device) of the two runs; present: [batch] int
 * (device). The runs reuse one workspace of uwb_presence_workspace(...)
 * bytes, one after the other on `stream`. */
size_t uwb_presence_workspace(int batch, int M, int N, const uwb_grid* grid, int beamformer,
                              const uwb_rule* rule, int decimation2);
int uwb_presence_batch(int batch, const float* traces, int M, int N, const float* antennas,
                       long long antenna_stride, const uwb_grid* grid, double v, double fs,
                       int window, int beamformer, const uwb_rule* rule, int decimation2,
                       void* workspace, size_t ws_bytes, uwb_result* out1, uwb_result* out2,
                       int* present, void* stream);

/* End-to-end localisation from HOST memory. traces_host [batch][M][N] and
 * antennas_host ([M][3], or [batch][...] with antenna_stride) live in host
 * memory (pinned memory lets the copies run asynchronously); out_host
 * receives `batch` uwb_result records in host memory. Only the window of
 * samples that some focal point of the grid can reach (round-trip delays over
 * the grid's bounding box, plus the window and a margin) is copied to the
 * device, with one strided copy; the localisation then runs as in
 * uwb_localize_batch, and the results are copied back. Everything is queued
 * on `stream`: host buffers must stay valid until it completes.
 * workspace: device memory of uwb_localize_host_workspace(...) bytes (it holds
 * the trace window, the antennas, the results and the search's scratch).
 * h2d_bytes (optional, host) receives the bytes copied to the device. */
size_t uwb_localize_host_workspace(int batch, const float* traces_host, int M, int N,
                                   const float* antennas_host, long long antenna_stride,
                                   const uwb_grid* grid, double v, double fs, int window,
                                   int beamformer, const uwb_rule* rule);
int uwb_localize_host(int batch, const float* traces_host, int M, int N,
                      const float* antennas_host, long long antenna_stride, const uwb_grid* grid,
                      double v, double fs, int window, int beamformer, const uwb_rule* rule,
                      void* workspace, size_t ws_bytes, uwb_result* out_host,
                      long long* h2d_bytes, void* stream);

/* uwb_localize_batch for callers that may not allocate device memory.
 *
 * Some callers cannot call cudaMalloc once they are running: acquisition
 * loops that must keep a fixed device-memory footprint and predictable
 * latency for the whole session, and plug-ins hosted by a framework that
 * owns every device allocation through its own pool. They cannot provide
 * the workspace uwb_localize_batch asks for, so this entry point takes none:
 * its scratch is a fixed array of UWB_NOALLOC_SCRATCH_BYTES (16 MiB) inside
 * the library, which every GPU that loads the library keeps until the
 * process exits. The paper has no counterpart to this; it is a deployment
 * convenience. Arguments and results are those of uwb_localize_batch.
 *  - It allocates nothing (no cudaMalloc, no cudaFree, no allocating
 *    library call); inputs and outputs still come from the caller.
 *  - Calls whose scratch need (uwb_localize_workspace for the same
 *    arguments) exceeds UWB_NOALLOC_SCRATCH_BYTES are rejected with
 *    UWB_ERR_WORKSPACE before any launch; split the batch instead.
 *  - The first call on a device looks up the address of that device's copy
 *    of the array and creates the library's events for that device (as the
 *    first call of any entry point does); make that first call before any
 *    stream capture.
 *  - Every call on a device uses the same array, and the array keeps the
 *    last call's contents (each call clears what it needs zeroed). Calls
 *    that overlap on the GPU (other streams, other host threads) race on
 *    it: serialise them, for example on one stream. */
#define UWB_NOALLOC_SCRATCH_BYTES (16u << 20)
int uwb_localize_batch_noalloc(int batch, const float* traces, int M, int N,
                               const float* antennas, long long antenna_stride,
                               const uwb_grid* grid, double v, double fs, int window,
                               int beamformer, const uwb_rule* rule, uwb_result* out,
                               float* image, void* stream);

/* Optional phase timing of uwb_localize / uwb_localize_batch (profiling aid).
 * While enabled, each call records CUDA events on its own stream around its
 * phases: 0 = decimated energy profile, 1 = segment selection and work
 * planning, 2 = final-region imaging, 3 = result decoding. The events add no
 * work to the kernels. Whether timing is on or not, the localisation calls
 * (batch, plan, learned, progressive) also open an NVTX range per phase
 * ("uwb decimated profile", "uwb selection", "uwb final region", "uwb
 * decode"; the learned call's first two are "uwb learned proposal" and "uwb
 * fallback selection") around the host calls that enqueue it, for a profiler
 * attached to the process (ncu --nvtx). uwb_phase_timing(1) switches timing on and discards
 * earlier records; uwb_phase_timing(0) switches it off. uwb_phase_times waits
 * for the recorded events, writes the summed milliseconds of each phase into
 * ms[0..3], forgets the records and returns how many calls they covered (or a
 * negative UWB_ERR_* code). */
int uwb_phase_timing(int enable);
int uwb_phase_times(double* ms);

/* Device-side status word shared by the image entry points: UWB_OK, or the
 * first error a kernel recorded (UWB_ERR_TIMEOUT). Synchronises the current
 * device; clear != 0 resets the word. Returns the word, or UWB_ERR_CUDA. */
int uwb_device_status(int clear);

/* Text of the last error of the calling thread ("" if none). */
const char* uwb_last_error(void);

/* Measurement aid for roofline fractions (no counterpart in the paper):
 * microbenchmarks of the two on-chip peaks the image kernels are bound by, on
 * the current device, synchronously. fp32_tflops: independent chains of paired
 * FP32 FMAs (2 FLOP per FMA); shared_wavefronts_per_s: conflict-free 32-bit
 * shared-memory loads, one 128-byte wavefront per warp instruction. Returns
 * UWB_OK or UWB_ERR_CUDA. */
int uwb_measure_peaks(double* fp32_tflops, double* shared_wavefronts_per_s);

/* Failure-detection self-check (no counterpart in the paper): shows that a
 * bounded device wait that runs out is reported and leaves the context usable.
 * One warp waits on a shared-memory mbarrier that nothing ever completes,
 * probing it with the bounded try-wait loop of the image kernels' staging wait
 * at most `probes` times (1 .. 2^24; each probe returns within a short
 * hardware time limit). The kernel then records UWB_ERR_TIMEOUT in the device
 * status word, exactly as a staging wait that runs out does, and returns.
 * Synchronous on the current device. Read the outcome with
 * uwb_device_status(); clear it there before further work. Returns UWB_OK
 * once the kernel has finished, UWB_ERR_ARG for probes outside 1 .. 2^24
 * (before any launch), or UWB_ERR_CUDA. */
int uwb_wait_selftest(int probes);

/* Progressive re-evaluation: a variant of uwb_localize_batch (the paper's
 * selection loop reads only the decimated profile). Iteration 1 is the
 * paper's. Every later iteration first images again the region being split on
 * its own lattice -- per axis at most the decimated lattice's point count c0,
 * step ceil(side / c0), centred like the decimated lattice -- and takes its
 * child choice from it: the variance of the region being split (sigma^2_{i-1}
 * of Eq. 5) and the children's Eq. 5 metrics. The Eq. 6-7 stopping rule keeps
 * reading the decimated profile, so consecutive iterations compare scatters
 * over one lattice; energies are divided by the profile maximum throughout.
 * Framing, final imaging and argmax as in uwb_localize_batch; arguments,
 * result records and errors as there, except points_evaluated, which also
 * counts every region lattice imaged. The loop runs as device kernels with
 * no host round trip (per iteration: one step kernel and one image pass). */
size_t uwb_localize_progressive_workspace(int batch, int M, int N, const uwb_grid* grid,
                                          int beamformer, const uwb_rule* rule);
int uwb_localize_progressive(int batch, const float* traces, int M, int N,
                             const float* antennas, long long antenna_stride,
                             const uwb_grid* grid, double v, double fs, int window,
                             int beamformer, const uwb_rule* rule, void* workspace,
                             size_t ws_bytes, uwb_result* results, void* stream);

/* ------------------------------------------------------------------------
 * Learned segment proposal. The paper has no counterpart: a small network
 * proposes the segments that Section III's ROI selection would otherwise pick
 * with the Eq. 5 metric, and Eq. 5 decides instead whenever the network is
 * not confident.
 *
 * Network: a 32 x 32 coarse DAS energy map (Eq. 1 + Eq. 3) of a square region
 * E is normalised, X0 = E / max E; three 3x3 zero-padded convolutions with 32
 * channels, bias and ReLU (1 -> 32 -> 32 -> 32 channels); the mean of the last
 * map over each of the 16 segments (4 x 4 squares of 8 x 8 map points,
 * s = 4 * row + column, row along grid axis 1); a shared linear head gives 16
 * segment scores z; confidence = the largest softmax probability of z.
 * Convolution weights are BF16 and feature maps are stored in BF16; every sum
 * accumulates in FP32 (the 32 -> 32 layers on the tensor cores).
 *
 * Parameters theta: UWB_CNN_PARAMS float32 values in the order
 *   W1[32][9], b1[32], W2[32][9][32], b2[32], W3[32][9][32], b3[32], wh[32], bh[1]
 * with W[c_out][tap][c_in] and tap = 3 (dy + 1) + (dx + 1), dy along grid axis
 * 1, dx along axis 0. The kernels read a packed copy (UWB_CNN_PACKED_BYTES,
 * 256-byte aligned device memory) made by uwb_cnn_pack or refreshed by
 * uwb_cnn_adam.
 *
 * The first call of uwb_cnn_forward, uwb_cnn_gradients, uwb_cnn_train_step
 * or uwb_localize_learned on a device runs a synchronous tensor-core
 * self-check (make it before any stream capture); if it fails, those calls
 * return UWB_ERR_UNSUPPORTED. All device pointers are caller-owned; the calls
 * are asynchronous on `stream`.
 * ---------------------------------------------------------------------- */
#define UWB_CNN_PARAMS 18849
#define UWB_CNN_PACKED_BYTES 38912

/* Runs (once per device) the tensor-core self-check: an exact integer-valued
 * BF16 GEMM through the descriptor and TMEM conventions the network uses.
 * *passed = 1 if the device reproduced it exactly. Returns UWB_OK or an error. */
int uwb_cnn_selftest(int* passed);

/* packed <- the kernels' copy of theta (device float[UWB_CNN_PARAMS]). */
int uwb_cnn_pack(const float* theta, void* packed, void* stream);

/* scores[b][16] <- segment scores of maps[b][32][32] (raw energies, row-major
 * [y][x]), b < batch. Non-finite map values set UWB_ERR_NONFINITE in the
 * device status word and read as 0. */
int uwb_cnn_forward(const void* packed, const float* maps, int batch, float* scores,
                    void* stream);

/* The per-map record of the forward pass, UWB_CNN_RECORD_BYTES per map (map b
 * at byte b * UWB_CNN_RECORD_BYTES). Map position (y, x) is buffer position
 * u = 34 + 33 y + x. Byte offsets within one map's record:
 *   0       X0 = E / max E, float, at 4 u
 *   5120    A1, BF16: channel c of position u at 5120 + (c / 8) * 19616 +
 *           16 u + 2 (c % 8)
 *   83584   A2, same layout (after uwb_cnn_gradients: G1, the BF16 gradient
 *           at layer 1's pre-activation)
 *   162048  A3, same layout (after uwb_cnn_gradients: G2, layer 2's)
 *   240512  segment means F[16][32], float
 *   242560  dz[16] = (softmax(z) - onehot(label)) / batch, float (written
 *           only when labels are given)
 * The same record is the first batch * UWB_CNN_RECORD_BYTES bytes of the
 * workspace of uwb_cnn_gradients. */
#define UWB_CNN_RECORD_BYTES 242688

/* uwb_cnn_forward that also writes the record above (record: 256-byte aligned
 * device memory of at least batch * UWB_CNN_RECORD_BYTES bytes), for checking
 * the network layer by layer. With labels (device int[batch] in [0, 16)) it
 * also writes dz and the mean cross-entropy into *loss (one device float,
 * zeroed first); labels may be NULL, and then loss is not used. */
int uwb_cnn_forward_record(const void* packed, const float* maps, const int* labels, int batch,
                           float* scores, float* loss, void* record, size_t record_bytes,
                           void* stream);

/* Workspace of uwb_cnn_train_step (a per-map record of the forward pass plus
 * one gradient vector); uwb_cnn_gradients needs batch * 242688 bytes. 0 for a
 * batch outside [1, 2^20]. */
size_t uwb_cnn_train_workspace(int batch);

/* Gradient of the mean cross-entropy of softmax(z) against labels[b] in
 * [0, 16) over the batch: grad (device float[UWB_CNN_PARAMS]) and loss (one
 * device float) are overwritten. The backward pass follows the chain rule of
 * the network with the gradient at each pre-activation rounded to BF16 before
 * it meets the weights (BF16 operands, FP32 sums, on the CUDA cores). The
 * workspace holds a per-map record of the forward pass; the backward pass
 * consumes it. workspace: 256-byte aligned device memory. */
int uwb_cnn_gradients(const void* packed, const float* maps, const int* labels, int batch,
                      float* grad, float* loss, void* workspace, size_t ws_bytes, void* stream);

/* Adam step `step` (from 1; beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected)
 * of theta with learning rate lr; m and v are its moment vectors (zero before
 * the first step). grad is consumed (zeroed) and packed refreshed. */
int uwb_cnn_adam(float* theta, float* m, float* v, float* grad, void* packed, int step, float lr,
                 void* stream);

/* uwb_cnn_gradients followed by uwb_cnn_adam, the gradient kept in the
 * workspace (uwb_cnn_train_workspace(batch) bytes). */
int uwb_cnn_train_step(float* theta, float* m, float* v, void* packed, const float* maps,
                       const int* labels, int batch, int step, float lr, float* loss,
                       void* workspace, size_t ws_bytes, void* stream);

/* Coarse DAS maps (Eq. 1 + Eq. 3 energies) of a square region per scan:
 * maps[b][ky][kx] at grid point (lo_x + o + step * kx, lo_y + o + step * ky),
 * step = side / 32, o = (step - 1) / 2. region_lo: device int[batch][2]
 * (x, y) per scan, or NULL for the region at (0, 0). Trace, antenna and grid
 * arguments as in uwb_localize_batch (2-D grids; side a multiple of 32 within
 * the grid). A region outside the grid sets UWB_ERR_ARG in the status word
 * and leaves its map at 0. workspace: uwb_coarse_maps_workspace(batch) bytes,
 * needed only with region_lo. */
size_t uwb_coarse_maps_workspace(int batch);
int uwb_coarse_maps(int batch, const float* traces, int M, int N, const float* antennas,
                    long long antenna_stride, const uwb_grid* grid, double v, double fs,
                    int window, const int* region_lo, int side, float* maps, void* workspace,
                    size_t ws_bytes, void* stream);

/* Localisation with the learned proposal, all on the device. For each of
 * `levels` levels (1..3) the scan's current square region (first the whole
 * grid) gets a coarse DAS map, the network scores its 16 segments, and the
 * scan descends into the best segment when the confidence is >= threshold.
 * After the last level the segment, framed by ceil(frame_num / frame_den *
 * side) points per side and clipped to the grid (Section III, sliding
 * framing), is imaged at full resolution with `beamformer` and its argmax
 * (lowest linear index on ties) is the location; stop_reason =
 * UWB_STOP_LEARNED, child[l] / metric_top[l] / box_lo[l] / box_hi[l] log the
 * segment, confidence and region of level l. A level below the threshold
 * hands the scan to the Eq. 5 framework of uwb_localize_batch (decimated
 * profile, ROI selection, final region) with the given rule. The grid must be
 * square and 2-D with a side divisible by 32 * 4^(levels - 1).
 * points_evaluated counts coarse-map, profile (fallback only) and final-region
 * points. workspace: uwb_localize_learned_workspace bytes, 256-byte aligned.
 * Phase timing records: 0 = proposal, 1 = fallback profile and selection,
 * 2 = final-region imaging, 3 = result decoding. */
size_t uwb_localize_learned_workspace(int batch, const uwb_grid* grid, const uwb_rule* rule);
int uwb_localize_learned(int batch, const float* traces, int M, int N, const float* antennas,
                         long long antenna_stride, const uwb_grid* grid, double v, double fs,
                         int window, int beamformer, const uwb_rule* rule, const void* packed,
                         float threshold, int levels, void* workspace, size_t ws_bytes,
                         uwb_result* results, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* UWB_H */
