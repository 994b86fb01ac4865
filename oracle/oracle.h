/*
 * FP64 CPU oracle for segment-search confocal UWB imaging
 * (Ettefagh, Moghaddam, Vahidian, "A Novel Low-Complexity Framework in
 * Ultra-Wideband Imaging for Breast Cancer Detection", arXiv:1709.02549).
 *
 * TEST INFRASTRUCTURE. This library exists to check the CUDA path. Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load it;
 * the product path never calls it and shares no code with it.
 *
 * Every function is a plain loop over the definition it cites, in double
 * precision, with no blocking, fusion or reordering beyond what the definition
 * states. OpenMP (when available) only splits independent focal points across
 * threads; each focal point's arithmetic is the same in any thread count.
 */
#ifndef UWB_ORACLE_H
#define UWB_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_ITERS 32

/* beamformers */
#define ORC_DAS 0
#define ORC_DMAS 1          /* pairwise products, Section II.B; literal i<j loop */

/* decimation modes, Section III "Spatial Decimation" */
#define ORC_DECIM_MANUAL 0
#define ORC_DECIM_AUTO 1

/* decision metrics, Section III "ROI Selection" */
#define ORC_METRIC_HYBRID 0   /* Eq. 5 */
#define ORC_METRIC_MEAN 1
#define ORC_METRIC_VARIANCE 2
#define ORC_METRIC_HYBRID_UNCLIPPED 3 /* Eq. 5 exactly as printed */

/* stop reasons */
#define ORC_STOP_NONE 0
#define ORC_STOP_METRIC 1     /* Eq. 6-7 rule failed */
#define ORC_STOP_MINSIZE 2    /* no child segment left to choose */
#define ORC_STOP_CAP 3        /* iteration cap */
#define ORC_STOP_NO_TARGET 4  /* all decimated energies are zero */

/* status */
#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_NONFINITE -4

/* Focal-point lattice: point idx (per axis) sits at origin + idx * pitch. */
typedef struct {
  int dim;
  int n[3];
  double origin[3];
  double pitch[3];
} orc_grid;

typedef struct {
  int mode;                   /* ORC_DECIM_MANUAL | ORC_DECIM_AUTO */
  int decimation;             /* manual factor D >= 1 */
  double min_tumor_diameter;  /* auto mode: smallest tumour to detect [m] */
  int metric;                 /* ORC_METRIC_* */
  int min_segment;            /* smallest child side, in full-resolution points */
  int frame_num, frame_den;   /* sliding-frame fraction of the child side */
  int max_iters;              /* 0 = ceil(log2(max grid side)) + 2 */
} orc_rule;

typedef struct {
  int status;
  int iters;                  /* accepted segmentations */
  int n_logged;               /* iterations performed (the last may be rejected) */
  int stop_reason;
  int decim;                  /* D */
  int offset[3];              /* decimated lattice offset per axis */
  int dcount[3];              /* decimated lattice points per axis */
  int roi_lo[3], roi_hi[3];   /* final region, full-resolution index box [lo, hi) */
  int loc_idx[3];             /* argmax of the final image, -1 if none */
  double loc_xyz[3];
  double peak;                /* image value at loc */
  double profile_max;         /* max of the decimated energies */
  long long points_evaluated; /* decimated points + final-region points */
  /* per performed iteration */
  int child[ORC_MAX_ITERS];
  int n_children[ORC_MAX_ITERS];     /* children that survived the filters */
  int box_lo[ORC_MAX_ITERS][3];
  int box_hi[ORC_MAX_ITERS][3];
  double metric_top[ORC_MAX_ITERS];
  double metric_gap[ORC_MAX_ITERS];  /* (top - runner-up) / |top|, 1e300 if alone */
  double between[ORC_MAX_ITERS];     /* B_i, Eq. 7 */
  double within[ORC_MAX_ITERS];      /* W_i, Eq. 6 */
  double stop_margin[ORC_MAX_ITERS]; /* robustness of the continue/stop outcome */
} orc_result;

/* Image over a box lattice of the focal grid (Eq. 1 with tau = 2|r-a|/v,
 * Eq. 3 for DAS, Section II.B for DMAS). Lattice point (kx,ky,kz) is grid
 * index lo + step * k; out is [cnt_z][cnt_y][cnt_x]. */
int orc_image(const float* traces, int M, int N, const float* antennas,
              const orc_grid* g, double v, double fs, int window, int beamformer,
              const int lo[3], const int step[3], const int cnt[3], double* out);

/* Multistatic image (Section II.A, Eq. 2 delays, Eq. 4 for DAS; DMAS over
 * pairs of channels): channel c is the echo sent by antenna chan[2c] and
 * received by antenna chan[2c+1], stored in traces[c][N]; its delay in
 * samples is (|r - a_tx| + |r - a_rx|) fs / v. Same lattice and output as
 * orc_image. */
int orc_image_multistatic(const float* traces, int C, int N, const int* chan,
                          const float* antennas, int M, const orc_grid* g, double v, double fs,
                          int window, int beamformer, const int lo[3], const int step[3],
                          const int cnt[3], double* out);

/* Spatial decimation factor, Section III (manual / automatic modes) and the
 * worked example of Section IV. */
int orc_decimation(const orc_rule* r, const orc_grid* g);

/* Offset of the decimated lattice along an axis of n points. */
int orc_lattice_offset(int n, int D);

/* ROI selection loop on a normalised decimated profile e[kz][ky][kx]
 * (Section III "ROI Selection", Eq. 5-7, sliding framing). Fills the
 * selection fields of res (not loc / peak / points_evaluated). */
int orc_select(const double* e, const orc_grid* g, const orc_rule* r, int D,
               orc_result* res);

/* Whole framework: decimated profile, normalisation, selection, final
 * full-resolution imaging of the region and its argmax (Section III). */
int orc_localize(const float* traces, int M, int N, const float* antennas,
                 const orc_grid* g, double v, double fs, int window, int beamformer,
                 const orc_rule* r, orc_result* res);

/* Tumour-presence test (Section IV, last paragraph): localise with the rule's
 * decimation factor and again with the manual factor `decimation2`; a tumour
 * is confirmed (returns 1) when both runs locate the same focal point, and
 * the scan is declared tumour-free (returns 0) when they disagree. res1 and
 * res2 receive the two runs. Negative on error. */
int orc_presence(const float* traces, int M, int N, const float* antennas, const orc_grid* g,
                 double v, double fs, int window, int beamformer, const orc_rule* r,
                 int decimation2, orc_result* res1, orc_result* res2);

/* The framework on a multistatic scan (channels as in orc_image_multistatic). */
int orc_localize_multistatic(const float* traces, int C, int N, const int* chan,
                             const float* antennas, int M, const orc_grid* g, double v,
                             double fs, int window, int beamformer, const orc_rule* r,
                             orc_result* res);

/* Progressive re-evaluation (a variant of Section III's ROI selection; the
 * paper's loop reads only the decimated profile). Iteration 1 is the paper's.
 * Every later iteration first images again the region being split, on the
 * lattice orc_region_lattice gives per axis with c0 = the decimated
 * lattice's point count on that axis, and takes its child choice from that
 * lattice: the region's variance (sigma^2_{i-1} of Eq. 5) and the children's
 * Eq. 5 metrics. The stopping rule (Eq. 6-7) keeps reading the decimated
 * profile, so that consecutive iterations compare scatters over one lattice.
 * Energies are divided by the maximum of the first profile throughout.
 * Framing, final imaging and argmax as in orc_localize; points_evaluated
 * counts every lattice point imaged plus the final region. */
int orc_localize_progressive(const float* traces, int M, int N, const float* antennas,
                             const orc_grid* g, double v, double fs, int window,
                             int beamformer, const orc_rule* r, orc_result* res);

/* Lattice of the index range [lo, hi) with at most c0 points: step
 * ceil((hi - lo) / c0), offset ((hi - lo - 1) mod step) / 2 from lo (the
 * centring rule of the decimated lattice), count (hi - lo - 1 - offset) / step
 * + 1. Writes the first index, the step and the count. */
void orc_region_lattice(int lo, int hi, int c0, int* first, int* step, int* cnt);

/* Trajectory replay, a test aid with no counterpart in the paper.
 *
 * Where two children score within rounding of each other (Eq. 5), or B_i and
 * W_i sit within rounding of B_{i-1} and W_{i-1} (Eq. 6-7), both outcomes are
 * correct, and an FP32 image may take the other one. A checker then needs the
 * oracle's answer along the path the other implementation took. An orc_path
 * makes the selection loop (Section III, ROI Selection) follow such a path:
 *  - iteration i (1-based, i <= n) takes child[i-1] when it is >= 0, instead
 *    of the argmax of the metric; the child must be a candidate (it survives
 *    the size and emptiness filters), else `error` is set to i and the call
 *    fails with ORC_ERR_ARG;
 *  - from the second iteration on, cont[i-1] >= 0 replaces the outcome of the
 *    Eq. 6-7 test: 1 continues, 0 stops with ORC_STOP_METRIC.
 * Everything else runs unchanged: every candidate's metric, the framing,
 * both scatters, the stop margins, the final region and its argmax. For each
 * performed iteration the loop records what it would have done itself
 * (own_child, own_cont) and how far the child it took is from its own best
 * (taken_gap = (best - taken) / |best|, 0 when they are the same child). The
 * result's child, box and metric_top entries describe the child taken;
 * metric_gap and stop_margin keep the oracle's own margins. */
typedef struct {
  int n;
  int child[ORC_MAX_ITERS];
  int cont[ORC_MAX_ITERS];
  /* written by the loop */
  int error;
  int own_child[ORC_MAX_ITERS];
  int own_cont[ORC_MAX_ITERS];        /* -1 at the first iteration (no test) */
  double taken_metric[ORC_MAX_ITERS];
  double taken_gap[ORC_MAX_ITERS];
} orc_path;

/* orc_select, orc_localize, orc_localize_multistatic and
 * orc_localize_progressive along a given path (path may be NULL: the
 * oracle's own choices, exactly as the functions without the suffix). */
int orc_select_path(const double* e, const orc_grid* g, const orc_rule* r, int D,
                    orc_path* path, orc_result* res);
int orc_localize_path(const float* traces, int M, int N, const float* antennas,
                      const orc_grid* g, double v, double fs, int window, int beamformer,
                      const orc_rule* r, orc_path* path, orc_result* res);
int orc_localize_multistatic_path(const float* traces, int C, int N, const int* chan,
                                  const float* antennas, int M, const orc_grid* g, double v,
                                  double fs, int window, int beamformer, const orc_rule* r,
                                  orc_path* path, orc_result* res);
int orc_localize_progressive_path(const float* traces, int M, int N, const float* antennas,
                                  const orc_grid* g, double v, double fs, int window,
                                  int beamformer, const orc_rule* r, orc_path* path,
                                  orc_result* res);

/* Eq. 5 hybrid metric for one candidate, weight clipped to [0, 1], and the
 * printed formula without the clip (exposed for the tests). */
double orc_hybrid_metric(double mean_i, double var_i, double var_prev);
double orc_hybrid_metric_unclipped(double mean_i, double var_i, double var_prev);

/* Eq. 6 / Eq. 7 for two scalar classes a and b (exposed for the tests). */
void orc_scatter(const double* a, int na, const double* b, int nb,
                 double* within, double* between);

int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
