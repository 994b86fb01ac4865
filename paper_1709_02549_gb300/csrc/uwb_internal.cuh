// Internal interfaces shared by the translation units of libuwb.so.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "uwb.h"

namespace uwb {

enum { BF_DAS = 0, BF_DMAS_ID = 1, BF_DMAS_LIT = 2 };

// Element type of the stored traces (arithmetic is float32 either way).
enum { DT_F32 = 0, DT_F16 = 1, DT_BF16 = 2 };
inline __host__ __device__ int dtype_bytes(int dt) { return dt == DT_F32 ? 4 : 2; }

// Everything the image kernel needs to know about one scan. Uniform batches
// derive it from ImgParams; ragged batches (scans of different antenna
// counts, trace lengths, grids) pass one per scan.
struct ScanDesc {
  const void* traces;   // first stored sample of trace row 0
  const float* ant;     // [M][3] antenna positions
  long long img_off;    // element offset of this scan's image in ImgParams::image
  long long cmp_off;    // element offset of this scan's compact profile
  int pitch;            // elements between trace rows
  int n_begin, N;       // stored samples [n_begin, n_begin + N); others read as 0
  int M, R;             // antennas, trace rows (R = M monostatic)
  int tma;              // ragged: index into ImgParams::tmaps (-1 = plain staging)
  float kscale;         // 2 fs / v
  float org[3], pit[3];
  int gn[3];
};

// A box lattice of the focal grid: lattice point k (per axis) is grid index
// lo + step * k, for 0 <= k < cnt. `tiles` = tiles of the image kernel's tile
// shape needed to cover it (lattice_tiles).
struct LatBox {
  int lo[3];
  int step[3];
  int cnt[3];
  int tiles;
};

// Tiles of the image kernel, one launch-wide kind. Linear tiles (tdim = {P,
// 0, 0}, P = focal points per CTA; the default): tile t holds the lattice's
// points t * P .. t * P + P - 1 in x-fastest order, so lattices whose sides
// are not multiples of a tile leave no partly empty warps but the last.
// Shaped tiles (tdim = powers of two per axis multiplying to P): tdim points
// per axis, warps of compact wdim blocks, which span fewer delay samples on
// coarse lattices.
__host__ __device__ inline bool tile_linear(const int tdim[3]) { return tdim[1] == 0; }

__host__ __device__ inline int lattice_tiles(const int cnt[3], const int tdim[3]) {
  if (cnt[0] <= 0 || cnt[1] <= 0 || cnt[2] <= 0) return 0;
  if (tile_linear(tdim)) {
    const long long n = static_cast<long long>(cnt[0]) * cnt[1] * cnt[2];
    return static_cast<int>((n + tdim[0] - 1) / tdim[0]);
  }
  long long t = 1;
  for (int a = 0; a < 3; ++a) t *= (cnt[a] + tdim[a] - 1) / tdim[a];
  return static_cast<int>(t);
}

// Everything the image kernels read. Scans of one launch share M, N, the grid
// and the lattice shape (uniform lattice) or each has its own box (per-scan
// lattices with a tile prefix sum, used for the final regions).
struct ImgParams {
  // Uniform batches: sample n of antenna i of scan s is traces[s * trace_stride
  // + i * pitch + (n - n_begin)] for n_begin <= n < n_begin + N, and 0 outside
  // (elements of type `dtype`).
  const void* traces;
  long long trace_stride;    // floats between scans
  int pitch;                 // floats between antenna rows
  int n_begin;               // sample index of the first stored sample
  const float* ant;          // [M][3] per scan
  long long ant_stride;      // floats between scans' antenna arrays (0 = shared)
  const int2* chan;          // multistatic: [R] (transmitter, receiver); else nullptr
  int R;                     // trace rows per scan: M (monostatic) or channels
  int B, M, N, W, h;
  float kscale;              // 2 fs / v: samples per metre of one-way path
  float org[3], pit[3];      // grid origin and pitch (float32)
  int gn[3];                 // grid points per axis
  long long gP;              // points per image
  LatBox uni;                // the lattice of every scan when boxes == nullptr
  const LatBox* boxes;       // per-scan lattices (device) or nullptr
  const int* prefix;         // [B+1] exclusive tile prefix when boxes != nullptr
  int tdim[3];               // tile shape, or {P, 0, 0} for linear tiles (tile_linear)
  int strip;                 // linear tiles of a 2-D box: > 1 = points numbered in strips
                             // of `strip` rows (column by column inside a strip), else
                             // row by row
  int wdim[3];               // warp sub-block extent of shaped tiles (product 32)
  int span;                  // samples staged per antenna (multiple of 4)
  int wpad;                  // window samples a thread may read (>= W, chunk multiple)
  int use_tma;               // stage with cp.async.bulk.tensor (else plain loads)
  float* image;              // [B][gP] or nullptr
  float* compact;            // [B][cnt0*cnt1*cnt2] or nullptr (uniform lattice)
  long long compact_stride;  // floats between scans in `compact`
  unsigned long long* keys;  // [B] argmax keys or nullptr
  int* status;               // device status word
  int* work;                 // tile counter, zero at launch (dynamic split), or nullptr
  int dtype;                 // DT_* of the traces
  const ScanDesc* descs;     // ragged batches: [B] per-scan descriptors (device), else nullptr
  const CUtensorMap* tmaps;  // ragged batches: per-scan tensor maps (device), or nullptr
  int Mcap, Rcap;            // largest M and R of the launch (shared-memory layout)
};

// Byte layout of the image kernel's dynamic shared memory:
//   [rows][span] float32 trace window (rows = R, or the literal kernel's
//   antenna block), [rows][span] raw 16-bit staging area (FP16/BF16 traces),
//   [Mcap] antennas (float4), (multistatic) [Rcap] channels, (literal)
//   [rows][threads] (offset, fraction) pairs, (multistatic) [Mcap][threads]
//   distances, the scan descriptor, an mbarrier, 32 reduction keys, 4 ints.
struct SmemLayout {
  size_t raw, ant, ch, nf, d, desc, bar, key, ints, total;
};

inline __host__ __device__ size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline __host__ __device__ SmemLayout image_smem_layout(int bf, int Mcap, int Rcap, int rows,
                                                        int span, int threads, bool ms,
                                                        int dtype) {
  SmemLayout L;
  const size_t window = static_cast<size_t>(rows) * span * 4;
  size_t off = align_up(window, 128);
  L.raw = off;
  // literal DMAS up to 64 antennas keeps a per-thread (offset, fraction)
  // table; the 32-antenna block form beyond recomputes delays instead
  const bool lit_table = bf == BF_DMAS_LIT && rows <= 64;
  if (dtype != DT_F32 && !lit_table) {
    // a 16-bit window lands in the upper half of the float window's area
    // (128-byte aligned for the copy) and is widened in place, front to back
    L.raw = align_up(static_cast<size_t>(rows) * span * 2, 128);
    const size_t end = L.raw + static_cast<size_t>(rows) * span * 2;
    off = align_up(end > window ? end : window, 128);
  }
  L.ant = off;
  off += static_cast<size_t>(Mcap) * 16;
  L.ch = off;
  if (ms) off += static_cast<size_t>(Rcap) * 8;
  if (lit_table && dtype != DT_F32) {
    // the table is written only after a staged window has been widened, so a
    // 16-bit window lands in the table (rows * span * 2 <= rows * threads * 8
    // bytes: span <= 256 <= 4 * threads; 128-byte aligned for the copy)
    off = align_up(off, 128);
    L.raw = off;
  }
  L.nf = off;
  if (lit_table) off += static_cast<size_t>(rows) * threads * 8;
  L.d = off;
  if (ms) off += static_cast<size_t>(Mcap) * threads * 4;
  off = align_up(off, 16);
  L.desc = off;
  off += align_up(sizeof(ScanDesc), 16);
  L.bar = off;
  off += 8;
  L.key = off;
  off += 32 * 8;
  L.ints = off;
  off += 4 * 4;
  L.total = off;
  return L;
}

// Per-scan decimated lattice and decision inputs (ragged batches).
struct SelScan {
  long long prof_off;        // element offset of the scan's profile
  int gn[3];                 // grid points per axis
  int off[3], step[3], cnt[3];  // decimated lattice
  int D, max_iters;
};

// Per-scan grid for decoding locations (ragged batches).
struct FinScan {
  int gn[3];
  double org[3], pit[3];
  long long Pd;              // decimated points
};

// Segment-selection inputs (one warp, or a quarter warp, per scan).
struct SelParams {
  const SelScan* scans;      // ragged: [B] (device), else nullptr
  const float* profile;      // [B][Pd] decimated energies, lattice order (x fastest)
  long long prof_stride;
  int B, dim;
  int gn[3];
  int off[3], step[3], cnt[3];   // decimated lattice
  int D;
  uwb_rule rule;
  int max_iters;
  int tdim[3];               // tile shape of the final-region image kernel
  const int* skip;           // per scan: nonzero = decided elsewhere, leave alone (or nullptr)
  LatBox* boxes;             // out: final region per scan
  uwb_result* out;           // out: results
};

// Per-scan state of the learned proposal across its levels.
struct LearnState {
  int lo[2];                 // current square region [lo, lo + side) per axis (x, y)
  int side;
  int fallback;              // 1: the Eq. 5 framework decides this scan
  int map_points;            // coarse-map points evaluated so far
};

// Per-scan state of the progressive re-evaluation loop.
struct ProgState {
  int Rlo[3], Rhi[3];        // current region
  double pmax;               // maximum of the decimated profile
  double B_prev, W_prev;     // Eq. 6-7 of the previous iteration
  long long points;          // focal points imaged so far (profile + region lattices)
  int active, iters, n_logged, stop;
};

// One iteration of the progressive loop for every scan (one warp per scan).
struct ProgParams {
  const float* profile;      // [B][Pd] decimated energies
  const float* lattice;      // [B][Pd] energies of each scan's region lattice (iteration >= 2)
  long long stride;          // Pd
  int B, dim;
  int gn[3];
  int off[3], step[3], cnt[3];  // decimated lattice
  int D, max_iters;
  uwb_rule rule;
  int tdim[3];               // tile shape of the image kernel
  ProgState* state;
  LatBox* next_boxes;        // out: region lattice of the next iteration (cnt 0: none)
  LatBox* final_boxes;       // out: final region of scans that stopped
  uwb_result* out;
};

struct FinishParams {
  const LearnState* learn;   // learned localisation: per-scan state, else nullptr
  const ProgState* prog;     // progressive loop: per-scan state, else nullptr
  const FinScan* scans;      // ragged: [B] (device), else nullptr
  const unsigned long long* keys;
  const LatBox* boxes;
  uwb_result* out;
  int B;
  int gn[3];
  double org[3], pit[3];
  long long Pd;
};

// Image-kernel launchers, one per beamformer; `v` selects the instance (window
// chunk WT for DAS / DMAS, antenna register block MMAX for literal DMAS).
// Each returns cudaGetLastError() after the launch.
// ms selects the multistatic instance (rows are channels).
cudaError_t launch_image_das(int v, bool ms, const ImgParams& p, const CUtensorMap* tmap,
                             int ctas, int threads, size_t smem, cudaStream_t st);
cudaError_t launch_image_dmas(int v, bool ms, const ImgParams& p, const CUtensorMap* tmap,
                              int ctas, int threads, size_t smem, cudaStream_t st);
cudaError_t launch_image_literal(int v, const ImgParams& p, const CUtensorMap* tmap, int ctas,
                                 int threads, size_t smem, cudaStream_t st);
// Sets the dynamic shared-memory limit of the instance and returns its
// resident CTAs per SM (0 on error).
int occupancy_image_das(int v, bool ms, bool rg, int threads, size_t smem);
int occupancy_image_dmas(int v, bool ms, bool rg, int threads, size_t smem);
int occupancy_image_literal(int v, bool rg, int threads, size_t smem);

cudaError_t launch_select(const SelParams& p, cudaStream_t st);
cudaError_t launch_prog_step(const ProgParams& p, int iteration, cudaStream_t st);
cudaError_t measure_peaks(int sms, double* tflops, double* wavefronts_per_s);
cudaError_t wait_selftest(int* status, long probes);
cudaError_t launch_plan(const LatBox* boxes, int* prefix, int B, cudaStream_t st);
cudaError_t launch_finish(const FinishParams& p, const int* status, cudaStream_t st);
cudaError_t launch_keys_to_index(unsigned long long* keys, int B, cudaStream_t st);
cudaError_t launch_presence(const uwb_result* a, const uwb_result* b, int* present, int B,
                            cudaStream_t st);

// ------------------------------------------------------ learned proposal
namespace cnn {
constexpr int MAP = 32;              // coarse map side
constexpr int CH = 32;               // channels
constexpr int TAPS = 9;              // 3 x 3
constexpr int SEG = 4;               // segments per axis
constexpr int SEGS = SEG * SEG;
constexpr int N_PARAMS = 18849;
// parameter vector offsets (floats): W1[32][9], b1, W2[32][9][32], b2, W3, b3, wh, bh
constexpr int TH_W1 = 0, TH_B1 = TH_W1 + CH * TAPS, TH_W2 = TH_B1 + CH;
constexpr int TH_B2 = TH_W2 + CH * TAPS * CH, TH_W3 = TH_B2 + CH;
constexpr int TH_B3 = TH_W3 + CH * TAPS * CH, TH_WH = TH_B3 + CH, TH_BH = TH_WH + CH;
static_assert(TH_BH + 1 == N_PARAMS, "parameter count");
// packed parameters (bytes): BF16 W1, W2, W3; FP32 b1, b2, b3, wh, bh
constexpr int PK_W1 = 0, PK_W2 = 1024, PK_W3 = PK_W2 + CH * TAPS * CH * 2;
constexpr int PK_F32 = PK_W3 + CH * TAPS * CH * 2, PK_BYTES = 38912;
static_assert(PK_F32 + (4 * CH + 1) * 4 <= PK_BYTES, "packed size");
// activation maps in shared memory: padded rows of Q positions, PAD0 zero
// positions first, U positions per 8-channel group of LBO_ACT bytes
constexpr int Q = MAP + 1, PAD0 = Q + 1, NPOS = MAP * Q, TILES = (NPOS + 127) / 128;
constexpr int U = 1224, LBO_ACT = U * 16 + 32, ACT_BYTES = 4 * LBO_ACT;
// per-map training record (bytes): X0 (float, U), A1, A2, A3 (padded BF16
// maps), segment means F[16][32], dz[16]
constexpr int SAVE_X0 = 0, SAVE_A1 = 5120, SAVE_A2 = SAVE_A1 + ACT_BYTES;
constexpr int SAVE_A3 = SAVE_A2 + ACT_BYTES, SAVE_F = SAVE_A3 + ACT_BYTES;
constexpr int SAVE_DZ = SAVE_F + SEGS * CH * 4, SAVE_BYTES = 242688;
static_assert(SAVE_DZ + SEGS * 4 <= SAVE_BYTES && U * 4 <= SAVE_A1, "training record");

struct LearnParams {
  int B, n, levels;
  float threshold;
  int frame_num, frame_den;
  const float* scores;       // [B][16]
  LearnState* state;         // [B]
  uwb_result* out;           // [B]
  LatBox* map_boxes;         // next level's coarse-map lattice (cnt 0: none)
  LatBox* final_boxes;       // final region of confident scans
  LatBox* prof_boxes;        // decimated lattice of fallback scans (cnt 0: none)
  int* learned;              // 1: the network decided the scan
  int doff[3], dstep[3], dcnt[3];  // the rule's decimated lattice
  int tdim_map[3], tdim_final[3];  // tile shapes of the map and final passes
};

size_t forward_smem();
size_t backward_smem();
size_t selftest_smem();
cudaError_t launch_selftest(const uint16_t* a, const uint16_t* b, float* d, int* status,
                            cudaStream_t st);
cudaError_t launch_forward(const void* packed, const float* maps, int B, float* scores,
                           const int* labels, void* save, float* loss, int* status, int ctas,
                           cudaStream_t st);
cudaError_t launch_backward(const void* packed, void* save, int B, float* grad, int ctas,
                            cudaStream_t st);
cudaError_t launch_pack(const float* theta, void* packed, cudaStream_t st);
// Adam constants, each rounded once to float from its double value:
// c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t)
struct AdamConsts {
  float lr, beta1, beta2, one_minus_beta1, one_minus_beta2, eps, c1, c2;
};
cudaError_t launch_adam(float* theta, float* m, float* v, float* grad, void* packed,
                        const AdamConsts& k, cudaStream_t st);
cudaError_t launch_decide(const LearnParams& p, int level, cudaStream_t st);
cudaError_t launch_region_boxes(const int* region_lo, int side, int n, int B, const int tdim[3],
                                LatBox* boxes, int* status, cudaStream_t st);
}  // namespace cnn

}  // namespace uwb
