// Internal interfaces shared by the translation units of libuwb.so.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "uwb.h"

namespace uwb {

enum { BF_DAS = 0, BF_DMAS_ID = 1, BF_DMAS_LIT = 2 };

// A box lattice of the focal grid: lattice point k (per axis) is grid index
// lo + step * k, for 0 <= k < cnt. `tiles` = tiles of the image kernel's tile
// shape needed to cover it.
struct LatBox {
  int lo[3];
  int step[3];
  int cnt[3];
  int tiles;
};

// Everything the image kernels read. Scans of one launch share M, N, the grid
// and the lattice shape (uniform lattice) or each has its own box (per-scan
// lattices with a tile prefix sum, used for the final regions).
struct ImgParams {
  // Sample n of antenna i of scan s is traces[s * trace_stride + i * pitch +
  // (n - n_begin)] for n_begin <= n < n_begin + N, and 0 outside.
  const float* traces;
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
  int tdim[3];               // tile extent in lattice points
  int wdim[3];               // warp sub-block extent (product 32)
  int span;                  // samples staged per antenna (multiple of 4)
  int wpad;                  // window samples a thread may read (>= W, chunk multiple)
  int use_tma;               // stage with cp.async.bulk.tensor (else plain loads)
  float* image;              // [B][gP] or nullptr
  float* compact;            // [B][cnt0*cnt1*cnt2] or nullptr (uniform lattice)
  long long compact_stride;  // floats between scans in `compact`
  unsigned long long* keys;  // [B] argmax keys or nullptr
  int* status;               // device status word
};

// Bytes of dynamic shared memory of the image kernel: [rows][span] traces
// (rows = M, or the antenna register block for literal DMAS), [M] antennas as
// float4, the literal kernel's [rows][threads] (offset, fraction) pairs, then
// an mbarrier, 32 reduction keys, 4 ints.
inline size_t image_smem_bytes(int bf, int M, int rows, int span, int threads, int R = 0,
                               bool ms = false) {
  const size_t ant_words = 4 * static_cast<size_t>(M);
  size_t b = (static_cast<size_t>(rows) * span + ant_words) * 4;
  if (ms) b += static_cast<size_t>(R) * 8 + static_cast<size_t>(M) * threads * 4;
  if (bf == BF_DMAS_LIT) b += static_cast<size_t>(rows) * threads * 8;
  b = (b + 7) & ~static_cast<size_t>(7);
  return b + 8 + 32 * 8 + 4 * 4;
}

// Segment-selection inputs (one warp per scan).
struct SelParams {
  const float* profile;      // [B][Pd] decimated energies, lattice order (x fastest)
  long long prof_stride;
  int B, dim;
  int gn[3];
  int off[3], step[3], cnt[3];   // decimated lattice
  int D;
  uwb_rule rule;
  int max_iters;
  int tdim[3];               // tile shape of the final-region image kernel
  LatBox* boxes;             // out: final region per scan
  uwb_result* out;           // out: results
};

struct FinishParams {
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
int occupancy_image_das(int v, bool ms, int threads, size_t smem);
int occupancy_image_dmas(int v, bool ms, int threads, size_t smem);
int occupancy_image_literal(int v, int threads, size_t smem);

cudaError_t launch_select(const SelParams& p, cudaStream_t st);
cudaError_t launch_plan(const LatBox* boxes, int* prefix, int B, cudaStream_t st);
cudaError_t launch_finish(const FinishParams& p, const int* status, cudaStream_t st);
cudaError_t launch_keys_to_index(unsigned long long* keys, int B, cudaStream_t st);
cudaError_t launch_presence(const uwb_result* a, const uwb_result* b, int* present, int B,
                            cudaStream_t st);

}  // namespace uwb
