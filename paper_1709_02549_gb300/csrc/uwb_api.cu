// C ABI of libuwb.so: argument checks, the spatial-decimation rule, workspace
// layout, TMA descriptor encoding, tile/warp shape choice and the launch
// sequence of the device-resident segment search.
#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>

#include "uwb_internal.cuh"

// Status word of the image entry points (they take no workspace); kernels
// record UWB_ERR_TIMEOUT here when a bounded staging wait runs out.
__device__ int g_uwb_status_word;

// Tile counters of the image kernel's dynamic work split, one per launch in
// flight (see take_counter).
constexpr int kCounterSlots = 64;
__device__ int g_uwb_tile_counters[kCounterSlots];

namespace uwb {
namespace {

thread_local char t_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_err, sizeof t_err, fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(UWB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

struct Device {
  bool ready = false;
  int sms = 0;
  int* status = nullptr;
  // tile counters: slot k is free once ev[k], recorded behind the last
  // launch that used it, has completed
  int* counters = nullptr;
  cudaEvent_t ev[kCounterSlots] = {};
  int next = 0;
  std::mutex counter_mu;
};

std::mutex g_mu;
Device g_devs[64];
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
bool g_encode_tried = false;

int device(Device** out) {
  int d = 0;
  cudaError_t e = cudaGetDevice(&d);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (d < 0 || d >= 64) return fail(UWB_ERR_UNSUPPORTED, "device ordinal %d", d);
  std::lock_guard<std::mutex> lk(g_mu);
  Device& dev = g_devs[d];
  if (!dev.ready) {
    e = cudaDeviceGetAttribute(&dev.sms, cudaDevAttrMultiProcessorCount, d);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&dev.status), g_uwb_status_word);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&dev.counters), g_uwb_tile_counters);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    // a slot whose event cannot be created is never used
    for (cudaEvent_t& ev : dev.ev)
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        ev = nullptr;
      }
    dev.ready = true;
  }
  if (!g_encode_tried) {
    g_encode_tried = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    else
      cudaGetLastError();
  }
  *out = &dev;
  return UWB_OK;
}

// ---- optional phase timing (events recorded on the caller's stream)
constexpr int kPhases = 4;
struct PhaseEvents {
  cudaEvent_t ev[kPhases + 1];
};
std::mutex g_timing_mu;
bool g_timing = false;
std::vector<PhaseEvents> g_phase_records;

void drop_records() {
  for (auto& r : g_phase_records)
    for (auto e : r.ev) cudaEventDestroy(e);
  g_phase_records.clear();
}

// Phase names of the NVTX ranges (a profiler attached to the process shows
// them; without one the calls return at once).
const char* const kLocalizePhases[kPhases] = {"uwb decimated profile", "uwb selection",
                                              "uwb final region", "uwb decode"};
const char* const kLearnedPhases[kPhases] = {"uwb learned proposal", "uwb fallback selection",
                                             "uwb final region", "uwb decode"};

// Events of one call (when timing is on) and an NVTX range per phase: mark()
// ends the phase that is open and opens the next.
struct PhaseTimer {
  PhaseEvents pe;
  bool on = false;
  int next = 0;
  int range = 0;  // NVTX ranges opened so far
  const char* const* names;
  explicit PhaseTimer(cudaStream_t st, const char* const* phase_names = kLocalizePhases)
      : names(phase_names), stream(st) {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    if (!g_timing) return;
    for (int i = 0; i <= kPhases; ++i)
      if (cudaEventCreate(&pe.ev[i]) != cudaSuccess) {
        for (int j = 0; j < i; ++j) cudaEventDestroy(pe.ev[j]);
        cudaGetLastError();
        return;
      }
    on = true;
  }
  void mark() {
    if (range > 0 && range <= kPhases) nvtxRangePop();
    if (range < kPhases) nvtxRangePushA(names[range]);
    ++range;
    if (on && next <= kPhases) cudaEventRecord(pe.ev[next++], stream);
  }
  void commit() {
    if (!on) return;
    std::lock_guard<std::mutex> lk(g_timing_mu);
    if (next == kPhases + 1) {
      g_phase_records.push_back(pe);
    } else {
      for (auto e : pe.ev) cudaEventDestroy(e);
    }
    on = false;
  }
  ~PhaseTimer() {
    if (range > 0 && range <= kPhases) nvtxRangePop();  // a call that left early
    if (on)
      for (auto e : pe.ev) cudaEventDestroy(e);
  }
  cudaStream_t stream;
};

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// Scans of one call: shared sizes and geometry.
struct Geo {
  int B, M, N, W, h;
  int R;              // trace rows per scan: M, or the multistatic channel count
  const int2* chan;   // multistatic channel table (device) or nullptr
  int pitch;    // floats between antenna rows of the trace array
  int n_begin;  // sample index of the first stored sample
  double v, fs;
  float kscale;
  uwb_grid g;
  long long P;
};

int check_common(int batch, const float* traces, int M, int N, const float* ant,
                 const uwb_grid* grid, double v, double fs, int window, Geo* geo) {
  if (batch < 1 || batch > (1 << 24)) return fail(UWB_ERR_ARG, "batch %d out of range", batch);
  if (!traces || !ant) return fail(UWB_ERR_ARG, "null traces or antennas");
  if (M < 1 || M > 4096) return fail(UWB_ERR_ARG, "antenna count M=%d out of [1, 4096]", M);
  if (N < 1) return fail(UWB_ERR_ARG, "trace length N=%d < 1", N);
  if (window < 1 || window > 4096) return fail(UWB_ERR_ARG, "window %d out of [1, 4096]", window);
  if (!finite_pos(v) || !finite_pos(fs)) return fail(UWB_ERR_ARG, "v and fs must be finite and > 0");
  if (!grid) return fail(UWB_ERR_ARG, "null grid");
  if (grid->dim != 2 && grid->dim != 3) return fail(UWB_ERR_ARG, "grid dim %d not 2 or 3", grid->dim);
  long long P = 1;
  for (int a = 0; a < 3; ++a) {
    if (grid->n[a] < 1) return fail(UWB_ERR_ARG, "grid n[%d] = %d < 1", a, grid->n[a]);
    if (!std::isfinite(grid->origin[a])) return fail(UWB_ERR_ARG, "grid origin not finite");
    if (a < grid->dim && !finite_pos(grid->pitch[a]))
      return fail(UWB_ERR_ARG, "grid pitch[%d] must be finite and > 0", a);
    P *= grid->n[a];
  }
  if (grid->dim == 2 && grid->n[2] != 1) return fail(UWB_ERR_ARG, "2-D grid needs n[2] == 1");
  // below 2^31 by more than a tile, so that every focal-point index of a
  // linear tile (tile * 256 + thread) stays a non-negative int
  if (P > 0x7FFFF000LL) return fail(UWB_ERR_ARG, "grid of %lld points exceeds 2^31 - 4096", P);
  const double ks = 2.0 * fs / v;
  if (!std::isfinite(static_cast<float>(ks))) return fail(UWB_ERR_ARG, "2 fs / v overflows float");
  geo->B = batch;
  geo->M = M;
  geo->N = N;
  geo->R = M;
  geo->chan = nullptr;
  geo->pitch = N;
  geo->n_begin = 0;
  geo->W = window;
  geo->h = window / 2;
  geo->v = v;
  geo->fs = fs;
  geo->kscale = static_cast<float>(ks);
  geo->g = *grid;
  if (grid->dim == 2) geo->g.pitch[2] = 1.0;
  geo->P = P;
  return UWB_OK;
}

struct Variant {
  int bf, v, threads;
  int tdim[3];
  int wpad;
  int rows;           // trace rows in shared memory
  size_t smem_budget; // shared memory per CTA the span is sized for
  bool ms;            // multistatic rows (channels)
  bool rg;            // launched with per-scan descriptors (ragged plans)
  int M, R;           // antennas, trace rows per scan
};

// Tile shapes chosen by uwb_autotune / uwb_set_tile_shape, per beamformer and
// dimensionality (0 = the built-in default).
std::mutex g_tile_mu;
int g_tile[3][4][3] = {};

bool tile_ok(int bf, const int t[3]) {
  if (t[0] == 0 && t[1] == 0 && t[2] == 0) return true;  // linear tiles
  const int points = bf == BF_DMAS_LIT ? 128 : 256;  // focal points per tile
  for (int a = 0; a < 3; ++a)
    if (t[a] < 1 || (t[a] & (t[a] - 1))) return false;  // powers of two
  return t[0] * t[1] * t[2] == points;
}

int var_points(const Variant& v);
int pick_span(const Variant& var, int M, int dtype = DT_F32);

int pick_variant(int bf, int M, int W, int dim, Variant* out, int R = -1) {
  Variant var;
  var.bf = bf;
  var.ms = R >= 0;
  var.rg = false;
  var.M = M;
  var.R = R >= 0 ? R : M;
  if (var.ms && bf == BF_DMAS_LIT)
    return fail(UWB_ERR_UNSUPPORTED, "literal-pair DMAS is built for monostatic data only");
  if (bf == BF_DMAS_LIT) {
    if (M > 96) return fail(UWB_ERR_UNSUPPORTED, "literal-pair DMAS supports M <= 96 (M=%d)", M);
    var.v = M <= 16 ? 16 : (M <= 32 ? 32 : (M <= 64 ? 64 : 96));
    // window samples go in fours (16-antenna block) or pairs
    var.wpad = var.v <= 16 ? (W + 3) / 4 * 4 : (W + 1) / 2 * 2;
    var.threads = 128;
    var.rows = var.v;
    // 4 CTAs (2 for the 64-antenna block, 3 for the 96-antenna block form)
    // per SM, each with the 1 KB the runtime reserves per CTA, fill the SM's
    // 228 KB
    var.smem_budget = var.v <= 32 ? 56 * 1024 : (var.v <= 64 ? 112 : 74) * 1024;
    var.tdim[0] = 128; var.tdim[1] = 0; var.tdim[2] = 0;  // linear tiles
  } else {
    // window chunk: the whole window up to 20 samples; longer windows go in
    // chunks of 16 (two focal points per thread) or 32 (multistatic)
    var.v = W <= 4 ? 4 : W <= 8 ? 8 : W <= 16 ? 16 : W <= 20 ? 20 : (var.ms ? 32 : 16);
    var.wpad = (W + var.v - 1) / var.v * var.v;
    // uniform monostatic: 128 threads of two focal points each (64 for few
    // trace rows, below); multistatic: 256 threads of two; ragged plans (see
    // use_ragged_shape): 256 threads of one
    var.threads = var.ms ? 256 : 128;
    var.rows = var.R;
    // window budget per CTA: the CTAs per SM of the launch shape share the
    // SM's 228 KB (point pairs: DAS 4, identity DMAS 3); multistatic rows are
    // M^2 channels: one CTA per SM with the span of up to 256 samples
    var.smem_budget = (var.ms ? 180 : (bf == BF_DAS ? 56 : 74)) * 1024;
    // linear tiles of the CTA's focal points (multistatic: 256 threads of two)
    var.tdim[0] = var.ms ? 512 : 256; var.tdim[1] = 0; var.tdim[2] = 0;
  }
  if (!var.ms) {  // tile shapes set by uwb_set_tile_shape / uwb_autotune (monostatic)
    std::lock_guard<std::mutex> lk(g_tile_mu);
    const int* t = g_tile[bf][dim];  // {0, 0, 0}: the default, linear tiles
    if (t[0] && (dim == 3 || t[2] == 1))
      for (int a = 0; a < 3; ++a) var.tdim[a] = t[a];
  }
  if (!var.ms && bf != BF_DMAS_LIT && tile_linear(var.tdim)) {
    // Few trace rows: CTAs of 64 threads (128-point tiles), twice as many per
    // SM, wherever half the shared-memory budget stages the same span. On
    // small final regions (a few hundred points per scan) each CTA spends a
    // good part of its time waiting on its own staging, tile grabs and
    // per-scan reductions; with more, smaller CTAs per SM those waits overlap
    // the other CTAs' tiles. The kernel takes its CTA size from the launch.
    Variant half = var;
    half.threads = 64;
    half.tdim[0] = 128;
    half.smem_budget = (bf == BF_DAS ? 27 : 37) * 1024;
    if (pick_span(half, M) == pick_span(var, M)) var = half;
  }
  *out = var;
  return UWB_OK;
}

// The coarse DAS maps of the learned proposal: 32 x 32 lattices with steps of
// 4 to 16 grid points. Shaped tiles 32 wide (8 rows, or 4 for CTAs of 64
// threads) divide them exactly and keep each warp's delay samples compact
// (fewer shared-memory bank conflicts than rows of 32 points), so they are
// used unless a shape was set for 2-D DAS.
int pick_map_variant(int M, int window, Variant* vm) {
  const int st = pick_variant(BF_DAS, M, window, 2, vm);
  if (st == UWB_OK && tile_linear(vm->tdim)) {
    vm->tdim[0] = 32; vm->tdim[1] = var_points(*vm) / 32; vm->tdim[2] = 1;
  }
  return st;
}

// Focal points of one CTA: uniform DAS and identity DMAS (monostatic and
// multistatic) evaluate two per thread; literal DMAS and ragged plans one.
int var_points(const Variant& v) {
  return v.threads * ((v.bf != BF_DMAS_LIT && !v.rg) ? 2 : 1);
}

// Ragged plans launch the per-scan-descriptor instances, which evaluate one
// focal point per thread (DAS and identity DMAS at 256 threads).
void use_ragged_shape(Variant* var) {
  var->rg = true;
  if (var->bf != BF_DMAS_LIT) {
    var->threads = 256;
    if (tile_linear(var->tdim)) var->tdim[0] = 256;  // one point per thread
    // those run 3 (DAS) or 2 (identity DMAS) CTAs per SM, each with the 1 KB
    // the runtime reserves: the rest of the SM's 228 KB sizes the staged span
    // of their (up to 96-row) windows
    var->smem_budget = (var->bf == BF_DAS ? 74 : 112) * 1024;
  }
}

// Warp sub-block shape: the one whose 32 focal points span the fewest delay
// samples (fewest shared-memory bank collisions), preferring wide x.
void pick_warp(const int tdim[3], const double delta[3], int wdim[3]) {
  if (tile_linear(tdim)) {  // a warp is 32 consecutive points
    wdim[0] = 32; wdim[1] = 1; wdim[2] = 1;
    return;
  }
  double best = 1e300;
  for (int wx = 32; wx >= 1; wx >>= 1)
    for (int wy = 32 / wx; wy >= 1; wy >>= 1) {
      const int wz = 32 / (wx * wy);
      if (wx * wy * wz != 32) continue;
      if (tdim[0] % wx || tdim[1] % wy || tdim[2] % wz) continue;
      const double cost = (wx - 1) * delta[0] + (wy - 1) * delta[1] + (wz - 1) * delta[2];
      if (cost < best - 1e-12) {
        best = cost;
        wdim[0] = wx; wdim[1] = wy; wdim[2] = wz;
      }
    }
}

// Samples staged per antenna: what the variant's shared-memory budget allows,
// at most one TMA box width (256), at least the window plus a margin.
int pick_span(const Variant& var, int M, int dtype) {
  // the largest span (a multiple of 8: 16-byte TMA rows for 16-bit traces too)
  // whose whole layout fits the budget
  int span = 256;
  while (span > 8 && image_smem_layout(var.bf, M, var.R, var.rows, span, var_points(var), var.ms,
                                       dtype).total > var.smem_budget)
    span -= 8;
  const int floor_span = (var.wpad + 8 + 7) & ~7;
  return span < floor_span ? floor_span : span;
}

// 3-D tensor map (sample, row, scan) over `scans` scans of `rows` trace rows,
// boxes of span x rows x 1. Returns 0 when TMA cannot serve the layout.
int encode_map(const void* traces, int dtype, int N, int pitch, int n_begin, int rows, int scans,
               int span, CUtensorMap* map) {
  memset(map, 0, sizeof *map);
  if (!g_encode) return 0;
  const int es = dtype_bytes(dtype);
  const int align = 16 / es;  // elements per 16 bytes
  if ((reinterpret_cast<uintptr_t>(traces) & 15) || (pitch % align) || (n_begin % align) ||
      N < 1 || rows > 256 || span > 256 || (span % align))
    return 0;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(N), static_cast<cuuint64_t>(rows),
                        static_cast<cuuint64_t>(scans)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(pitch) * es,
                           static_cast<cuuint64_t>(pitch) * rows * es};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(span), static_cast<cuuint32_t>(rows), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapDataType dt = dtype == DT_F32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : dtype == DT_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                   : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  CUresult r = g_encode(map, dt, 3, const_cast<void*>(traces), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 1 : 0;
}

int encode_traces(const Geo& geo, const float* traces, int span, CUtensorMap* map) {
  return encode_map(traces, DT_F32, geo.N, geo.pitch, geo.n_begin, geo.R, geo.B, span, map);
}

// Resident CTAs per SM of a kernel instance at a shared-memory size; cached
// per device, so that calls after the first (for example inside a CUDA-graph
// capture) query nothing and change no attribute.
struct OccKey {
  int dev, bf, v, ms, rg, threads;
  size_t smem;
  bool operator==(const OccKey& o) const {
    return dev == o.dev && bf == o.bf && v == o.v && ms == o.ms && rg == o.rg &&
           threads == o.threads && smem == o.smem;
  }
};
std::mutex g_occ_mu;
std::vector<std::pair<OccKey, int>> g_occ;

int occupancy(const Variant& var, size_t smem) {
  int d = 0;
  cudaGetDevice(&d);
  const OccKey key{d, var.bf, var.v, var.ms ? 1 : 0, var.rg ? 1 : 0, var.threads, smem};
  {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    for (const auto& kv : g_occ)
      if (kv.first == key) return kv.second;
  }
  int occ;
  switch (var.bf) {
    case BF_DAS: occ = occupancy_image_das(var.v, var.ms, var.rg, var.threads, smem); break;
    case BF_DMAS_ID: occ = occupancy_image_dmas(var.v, var.ms, var.rg, var.threads, smem); break;
    default: occ = occupancy_image_literal(var.v, var.rg, var.threads, smem); break;
  }
  if (occ > 0) {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    g_occ.emplace_back(key, occ);
  }
  return occ;
}

cudaError_t launch(const Variant& var, const ImgParams& p, const CUtensorMap* map, int ctas,
                   size_t smem, cudaStream_t st) {
  switch (var.bf) {
    case BF_DAS: return launch_image_das(var.v, var.ms, p, map, ctas, var.threads, smem, st);
    case BF_DMAS_ID:
      return launch_image_dmas(var.v, var.ms, p, map, ctas, var.threads, smem, st);
    default: return launch_image_literal(var.v, p, map, ctas, var.threads, smem, st);
  }
}


ImgParams base_params(const Geo& geo, const float* traces, const float* ant,
                      long long ant_stride, const Variant& var, int span, int use_tma,
                      int* status) {
  ImgParams p;
  memset(&p, 0, sizeof p);
  p.traces = traces;
  p.trace_stride = static_cast<long long>(geo.R) * geo.pitch;
  p.R = geo.R;
  p.chan = geo.chan;
  p.pitch = geo.pitch;
  p.n_begin = geo.n_begin;
  p.ant = ant;
  p.ant_stride = ant_stride;
  p.B = geo.B;
  p.M = geo.M;
  p.N = geo.N;
  p.W = geo.W;
  p.h = geo.h;
  p.kscale = geo.kscale;
  for (int a = 0; a < 3; ++a) {
    p.org[a] = static_cast<float>(geo.g.origin[a]);
    p.pit[a] = static_cast<float>(geo.g.pitch[a]);
    p.gn[a] = geo.g.n[a];
    p.tdim[a] = var.tdim[a];
  }
  p.gP = geo.P;
  p.dtype = DT_F32;
  p.Mcap = geo.M;
  p.Rcap = geo.R;
  p.span = span;
  p.wpad = var.wpad;
  p.use_tma = use_tma;
  p.status = status;
  return p;
}

// A free tile-counter slot of the device, or -1. Called with counter_mu held.
// The caller zeroes the slot on its stream, launches, and records ev[slot]
// behind the launch before releasing the lock, so a slot never serves two
// launches at once. While `st` is being captured into a graph no slot is
// taken (a captured launch would replay with one slot forever): the kernel
// then splits its tiles statically.
int take_counter(Device& dev, cudaStream_t st) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  if (cap != cudaStreamCaptureStatusNone) return -1;
  for (int k = 0; k < kCounterSlots; ++k) {
    const int slot = (dev.next + k) % kCounterSlots;
    if (!dev.ev[slot]) continue;
    const cudaError_t q = cudaEventQuery(dev.ev[slot]);  // an unrecorded event is complete
    if (q == cudaErrorNotReady) {
      if (cudaPeekAtLastError() == cudaErrorNotReady) cudaGetLastError();
      continue;
    }
    if (q != cudaSuccess) return -1;
    dev.next = slot + 1;
    return slot;
  }
  return -1;
}

// Launches the image kernel with a zeroed tile counter when one is free (the
// kernel then balances its tiles dynamically where it has enough of them),
// else with the static split. The counter evens out CTAs that share an SM;
// with one CTA per SM (per_sm == 1, the multistatic instances) the static
// split measured 2-4 % faster. Tile counts near 2^31 keep the static split.
// A call that owns a counter in its workspace (own_ctr, zeroed on the
// launch's stream before the launch) uses it instead of the pool: then a
// launch captured into a CUDA graph keeps the dynamic split, since every
// replay zeroes the counter again.
cudaError_t launch_balanced(Device& dev, const Variant& var, ImgParams& p, const CUtensorMap* map,
                            int ctas, int per_sm, size_t smem, long long work_bound,
                            cudaStream_t st, int* own_ctr = nullptr) {
  const bool balance = per_sm >= 2 && work_bound < (1LL << 30);
  if (own_ctr) {
    p.work = balance ? own_ctr : nullptr;
    return launch(var, p, map, ctas, smem, st);
  }
  std::lock_guard<std::mutex> lk(dev.counter_mu);
  const int slot = balance ? take_counter(dev, st) : -1;
  p.work = nullptr;
  if (slot >= 0) {
    const cudaError_t e = cudaMemsetAsync(dev.counters + slot, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    p.work = dev.counters + slot;
  }
  const cudaError_t e = launch(var, p, map, ctas, smem, st);
  if (e != cudaSuccess) return e;
  if (slot >= 0) return cudaEventRecord(dev.ev[slot], st);
  return cudaSuccess;
}

int run_image_kernel(Device& dev, const Variant& var, ImgParams& p, const CUtensorMap* map,
                     long long work_bound, const double step[3], cudaStream_t st,
                     int* own_ctr = nullptr) {
  double delta[3];
  for (int a = 0; a < 3; ++a) delta[a] = step[a] * p.pit[a] * p.kscale;
  if (p.gn[2] == 1) delta[2] = 1e9;  // keep warps flat in 2-D
  pick_warp(var.tdim, delta, p.wdim);
  // Linear tiles of a 2-D lattice whose delay changes by about a sample or
  // more per point: a row of 32 points would span 32+ samples and two lanes
  // would read words 32 apart (one shared-memory bank); strips of 4 rows
  // make each warp an 8 x 4 block spanning 7 dx + 3 dy samples (fewer than
  // 32 up to 3.2 samples per point). The 64 x 64 workload's final regions
  // (1.56 samples per point) had 20.8 M bank conflicts on 68.4 M wavefronts.
  const double dmax = std::fmax(delta[0], p.gn[2] == 1 ? delta[1] : 1e9);
  p.strip = (tile_linear(var.tdim) && p.gn[2] == 1 && dmax > 0.9 && dmax <= 3.2) ? 4 : 0;
  const size_t smem = image_smem_layout(var.bf, p.Mcap, p.Rcap, var.rows, p.span, var_points(var),
                                        var.ms, p.dtype).total;
  const int occ = occupancy(var, smem);
  if (occ < 1) return fail(UWB_ERR_UNSUPPORTED, "image kernel cannot launch with %zu B of shared memory", smem);
  long long ctas = static_cast<long long>(dev.sms) * occ;
  if (work_bound < ctas) ctas = work_bound;
  if (ctas < 1) return UWB_OK;
  cudaError_t e = launch_balanced(dev, var, p, map, static_cast<int>(ctas), occ, smem,
                                  work_bound, st, own_ctr);
  if (e != cudaSuccess) return cuda_fail(e, "image kernel launch");
  return UWB_OK;
}

int bf_of(int beamformer) {
  switch (beamformer) {
    case UWB_DAS: return BF_DAS;
    case UWB_DMAS: return BF_DMAS_ID;
    case UWB_DMAS_LITERAL: return BF_DMAS_LIT;
    default: return -1;
  }
}

int image_impl(int batch, int beamformer, const float* traces, int M, int N, const float* ant,
               long long ant_stride, const uwb_grid* grid, double v, double fs, int window,
               float* image, long long* peak_index, void* stream, int R = -1,
               const int* channels = nullptr) {
  Geo geo;
  int st = check_common(batch, traces, M, N, ant, grid, v, fs, window, &geo);
  if (st) return st;
  if (R >= 0) {
    if (R < 1 || R > 4096 || !channels) return fail(UWB_ERR_ARG, "multistatic needs 1..4096 channels");
    geo.R = R;
    geo.chan = reinterpret_cast<const int2*>(channels);
  }
  if (!image) return fail(UWB_ERR_ARG, "null image");
  if (ant_stride < 0) return fail(UWB_ERR_ARG, "negative antenna stride");
  const int bf = bf_of(beamformer);
  if (bf < 0) return fail(UWB_ERR_ARG, "unknown beamformer %d", beamformer);
  Variant var;
  if ((st = pick_variant(bf, M, window, grid->dim, &var, geo.chan ? geo.R : -1))) return st;
  Device* dev;
  if ((st = device(&dev))) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const int span = pick_span(var, M);
  CUtensorMap map;
  const int use_tma = encode_traces(geo, traces, span, &map);
  ImgParams p = base_params(geo, traces, ant, ant_stride, var, span, use_tma, dev->status);
  for (int a = 0; a < 3; ++a) {
    p.uni.lo[a] = 0;
    p.uni.step[a] = 1;
    p.uni.cnt[a] = geo.g.n[a];
  }
  p.uni.tiles = lattice_tiles(p.uni.cnt, var.tdim);
  p.image = image;
  p.keys = reinterpret_cast<unsigned long long*>(peak_index);
  cudaError_t e;
  if (peak_index) {
    e = cudaMemsetAsync(peak_index, 0, sizeof(long long) * batch, cs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  }
  const double step[3] = {1, 1, 1};
  if ((st = run_image_kernel(*dev, var, p, &map, static_cast<long long>(batch) * p.uni.tiles,
                             step, cs)))
    return st;
  if (peak_index) {
    e = launch_keys_to_index(p.keys, batch, cs);
    if (e != cudaSuccess) return cuda_fail(e, "argmax decode launch");
  }
  return UWB_OK;
}

int check_rule(const uwb_rule* r) {
  if (!r) return fail(UWB_ERR_ARG, "null rule");
  if (r->mode != UWB_DECIM_MANUAL && r->mode != UWB_DECIM_AUTO)
    return fail(UWB_ERR_ARG, "unknown decimation mode %d", r->mode);
  if (r->mode == UWB_DECIM_MANUAL && r->decimation < 1)
    return fail(UWB_ERR_ARG, "manual decimation %d < 1", r->decimation);
  if (r->mode == UWB_DECIM_AUTO && !finite_pos(r->min_tumor_diameter))
    return fail(UWB_ERR_ARG, "min_tumor_diameter must be finite and > 0");
  if (r->metric < UWB_METRIC_HYBRID || r->metric > UWB_METRIC_HYBRID_UNCLIPPED)
    return fail(UWB_ERR_ARG, "unknown metric %d", r->metric);
  if (r->min_segment < 1) return fail(UWB_ERR_ARG, "min_segment %d < 1", r->min_segment);
  if (r->frame_num < 0 || r->frame_den < 1 || r->frame_num > 1000000)
    return fail(UWB_ERR_ARG, "framing %d/%d invalid", r->frame_num, r->frame_den);
  if (r->max_iters < 0 || r->max_iters > UWB_MAX_ITERS)
    return fail(UWB_ERR_ARG, "max_iters %d out of [0, %d]", r->max_iters, UWB_MAX_ITERS);
  return UWB_OK;
}

// Section III: manual factor as given; automatic factor spaces the decimated
// points by the side of the square inscribed in the smallest tumour to find
// (d / sqrt 2), in units of the finest pitch (Section IV: 1 cm at 1 mm -> 7).
int decimation_of(const uwb_grid& g, const uwb_rule& r) {
  if (r.mode == UWB_DECIM_MANUAL) return r.decimation;
  double res = g.pitch[0];
  for (int a = 1; a < g.dim; ++a) res = std::fmin(res, g.pitch[a]);
  const double q = std::floor(r.min_tumor_diameter / std::sqrt(2.0) / res + 1e-9);
  if (!(q >= 1.0)) return 1;
  return q > 1e9 ? 1000000000 : static_cast<int>(q);
}

struct Decim {
  int D, off[3], step[3], cnt[3];
  long long Pd;
  int max_iters;
};

Decim decimate(const uwb_grid& g, const uwb_rule& r) {
  Decim d;
  d.D = decimation_of(g, r);
  d.Pd = 1;
  int nmax = 1;
  for (int a = 0; a < 3; ++a) {
    if (a < g.dim) {
      d.off[a] = ((g.n[a] - 1) % d.D) / 2;  // centred lattice
      d.step[a] = d.D;
      d.cnt[a] = (g.n[a] - 1 - d.off[a]) / d.D + 1;
      nmax = g.n[a] > nmax ? g.n[a] : nmax;
    } else {
      d.off[a] = 0;
      d.step[a] = 1;
      d.cnt[a] = g.n[a];
    }
    d.Pd *= d.cnt[a];
  }
  int lg = 0;
  while ((1LL << lg) < nmax) ++lg;
  d.max_iters = r.max_iters > 0 ? r.max_iters : lg + 2;
  if (d.max_iters > UWB_MAX_ITERS) d.max_iters = UWB_MAX_ITERS;
  return d;
}

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

struct WsLayout {
  size_t keys, status, counters, profile, boxes, prefix, total;
};

// Tile counters a localisation owns in its workspace: one per image pass.
constexpr int kWsCounters = 2;

WsLayout ws_layout(int B, long long Pd) {
  WsLayout w;
  size_t off = 0;
  w.keys = off;
  off += static_cast<size_t>(B) * 8;       // argmax keys ...
  w.status = off;                           // ... followed by the status word
  w.counters = off + 4;                     // and the passes' tile counters
  off = align256(off + 4 + 4 * kWsCounters);
  w.profile = off;
  off += align256(static_cast<size_t>(B) * static_cast<size_t>(Pd) * 4);
  w.boxes = off;
  off += align256(static_cast<size_t>(B) * sizeof(LatBox));
  w.prefix = off;
  off += align256(static_cast<size_t>(B + 1) * 4);
  w.total = off;
  return w;
}

int localize_core(const Geo& geo, const float* traces, const float* ant, long long ant_stride,
                  int beamformer, const uwb_rule* rule, void* workspace, size_t ws_bytes,
                  uwb_result* out, float* image, void* stream);

int localize_impl(int batch, const float* traces, int M, int N, const float* ant,
                  long long ant_stride, const uwb_grid* grid, double v, double fs, int window,
                  int beamformer, const uwb_rule* rule, void* workspace, size_t ws_bytes,
                  uwb_result* out, float* image, void* stream, int R = -1,
                  const int* channels = nullptr) {
  Geo geo;
  int st = check_common(batch, traces, M, N, ant, grid, v, fs, window, &geo);
  if (st) return st;
  if (R >= 0) {
    if (R < 1 || R > 4096 || !channels) return fail(UWB_ERR_ARG, "multistatic needs 1..4096 channels");
    geo.R = R;
    geo.chan = reinterpret_cast<const int2*>(channels);
  }
  if ((st = check_rule(rule))) return st;
  if (!out) return fail(UWB_ERR_ARG, "null result array");
  if (ant_stride < 0) return fail(UWB_ERR_ARG, "negative antenna stride");
  if (bf_of(beamformer) < 0) return fail(UWB_ERR_ARG, "unknown beamformer %d", beamformer);
  return localize_core(geo, traces, ant, ant_stride, beamformer, rule, workspace, ws_bytes, out,
                       image, stream);
}

// The device-resident search on validated arguments (traces as described by
// geo's N / pitch / n_begin).
int localize_core(const Geo& geo, const float* traces, const float* ant, long long ant_stride,
                  int beamformer, const uwb_rule* rule, void* workspace, size_t ws_bytes,
                  uwb_result* out, float* image, void* stream) {
  int st;
  const int batch = geo.B, M = geo.M, window = geo.W;
  const int bf = bf_of(beamformer);
  Variant var;
  if ((st = pick_variant(bf, M, window, geo.g.dim, &var, geo.chan ? geo.R : -1))) return st;
  const Decim dc = decimate(geo.g, *rule);
  const WsLayout wl = ws_layout(batch, dc.Pd);
  if (!workspace) return fail(UWB_ERR_WORKSPACE, "null workspace");
  if (reinterpret_cast<uintptr_t>(workspace) & 255)
    return fail(UWB_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (ws_bytes < wl.total)
    return fail(UWB_ERR_WORKSPACE, "workspace of %zu bytes < %zu needed", ws_bytes, wl.total);
  Device* dev;
  if ((st = device(&dev))) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  auto* keys = reinterpret_cast<unsigned long long*>(ws + wl.keys);
  auto* status = reinterpret_cast<int*>(ws + wl.status);
  auto* profile = reinterpret_cast<float*>(ws + wl.profile);
  auto* boxes = reinterpret_cast<LatBox*>(ws + wl.boxes);
  auto* prefix = reinterpret_cast<int*>(ws + wl.prefix);
  auto* counters = reinterpret_cast<int*>(ws + wl.counters);

  // keys, status word and tile counters start at zero
  cudaError_t e = cudaMemsetAsync(ws + wl.keys, 0, wl.counters + 4 * kWsCounters - wl.keys, cs);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");

  const int span = pick_span(var, M);
  CUtensorMap map;
  const int use_tma = encode_traces(geo, traces, span, &map);
  PhaseTimer timer(cs);
  timer.mark();

  // 1. energies of the decimated lattice (Section III, "Spatial Decimation")
  ImgParams p1 = base_params(geo, traces, ant, ant_stride, var, span, use_tma, status);
  for (int a = 0; a < 3; ++a) {
    p1.uni.lo[a] = dc.off[a];
    p1.uni.step[a] = dc.step[a];
    p1.uni.cnt[a] = dc.cnt[a];
  }
  p1.uni.tiles = lattice_tiles(p1.uni.cnt, var.tdim);
  p1.compact = profile;
  p1.compact_stride = dc.Pd;
  p1.image = image;
  const double dstep[3] = {static_cast<double>(dc.step[0]), static_cast<double>(dc.step[1]),
                           static_cast<double>(dc.step[2])};
  if ((st = run_image_kernel(*dev, var, p1, &map,
                             static_cast<long long>(batch) * p1.uni.tiles, dstep, cs,
                             counters)))
    return st;

  timer.mark();

  // 2. ROI selection loop (Section III, "ROI Selection"), a warp or a quarter warp per scan
  SelParams sp;
  memset(&sp, 0, sizeof sp);
  sp.profile = profile;
  sp.prof_stride = dc.Pd;
  sp.B = batch;
  sp.dim = geo.g.dim;
  for (int a = 0; a < 3; ++a) {
    sp.gn[a] = geo.g.n[a];
    sp.off[a] = dc.off[a];
    sp.step[a] = dc.step[a];
    sp.cnt[a] = dc.cnt[a];
    sp.tdim[a] = var.tdim[a];
  }
  sp.D = dc.D;
  sp.rule = *rule;
  sp.max_iters = dc.max_iters;
  sp.boxes = boxes;
  sp.out = out;
  if ((e = launch_select(sp, cs)) != cudaSuccess) return cuda_fail(e, "select launch");
  if ((e = launch_plan(boxes, prefix, batch, cs)) != cudaSuccess) return cuda_fail(e, "plan launch");

  timer.mark();

  // 3. final imaging of each scan's region at full resolution + argmax
  ImgParams p2 = base_params(geo, traces, ant, ant_stride, var, span, use_tma, status);
  p2.boxes = boxes;
  p2.prefix = prefix;
  p2.uni.tiles = 1;
  p2.keys = keys;
  p2.image = image;
  int full_cnt[3] = {geo.g.n[0], geo.g.n[1], geo.g.n[2]};
  const double step1[3] = {1, 1, 1};
  if ((st = run_image_kernel(*dev, var, p2, &map,
                             static_cast<long long>(batch) * lattice_tiles(full_cnt, var.tdim), step1,
                             cs, counters + 1)))
    return st;

  timer.mark();

  FinishParams fp;
  memset(&fp, 0, sizeof fp);
  fp.keys = keys;
  fp.boxes = boxes;
  fp.out = out;
  fp.B = batch;
  for (int a = 0; a < 3; ++a) {
    fp.gn[a] = geo.g.n[a];
    fp.org[a] = geo.g.origin[a];
    fp.pit[a] = geo.g.pitch[a];
  }
  fp.Pd = dc.Pd;
  if ((e = launch_finish(fp, status, cs)) != cudaSuccess) return cuda_fail(e, "finish launch");
  timer.mark();
  timer.commit();
  return UWB_OK;
}

// ---- host-buffer localisation: only the reachable sample window travels

// Samples [w0, w0 + len) of every trace that any focal point of the grid can
// read (round-trip delays over the grid's bounding box, the centred window,
// its padding, and a margin), clipped to the recorded trace and aligned for
// the tensor copies.
struct HostWindow {
  int w0, len, pitch;
};

HostWindow reachable_window(const Geo& geo, const float* ant_host, long long ant_stride) {
  double bmin[3], bmax[3];
  for (int a = 0; a < 3; ++a) {
    const double p0 = geo.g.origin[a];
    const double p1 = geo.g.origin[a] + (geo.g.n[a] - 1) * geo.g.pitch[a];
    bmin[a] = std::fmin(p0, p1);
    bmax[a] = std::fmax(p0, p1);
  }
  const double ks = 2.0 * geo.fs / geo.v;
  const long long scans = ant_stride ? geo.B : 1;
  double umin = 1e300, umax = -1e300;
  for (long long s = 0; s < scans; ++s)
    for (int i = 0; i < geo.M; ++i) {
      const float* a = ant_host + s * ant_stride + 3 * i;
      double dn2 = 0.0, df2 = 0.0;
      for (int k = 0; k < 3; ++k) {
        const double av = a[k];
        const double dn = av - std::fmin(std::fmax(av, bmin[k]), bmax[k]);
        const double df = std::fmax(std::fabs(av - bmin[k]), std::fabs(av - bmax[k]));
        dn2 += dn * dn;
        df2 += df * df;
      }
      umin = std::fmin(umin, std::sqrt(dn2) * ks);
      umax = std::fmax(umax, std::sqrt(df2) * ks);
    }
  // every kernel variant reads at most W + 32 samples past floor(u - h)
  const double lo = std::floor(umin - geo.h) - 8.0;
  const double hi = std::floor(umax - geo.h) + geo.W + 32 + 8.0;
  long long w0 = lo < 0 ? 0 : static_cast<long long>(lo);
  long long w1 = hi > geo.N ? geo.N : static_cast<long long>(hi);
  w0 &= ~3LL;
  if (w1 < w0) w1 = w0;
  HostWindow w;
  w.w0 = static_cast<int>(w0);
  w.len = static_cast<int>(w1 - w0);
  w.pitch = (w.len + 3) & ~3;
  if (w.pitch < 4) w.pitch = 4;
  return w;
}

struct HostLayout {
  size_t traces, ants, results, local, total;
};

HostLayout host_layout(const Geo& geo, const HostWindow& w, long long ant_stride,
                       const uwb_rule& rule) {
  HostLayout h;
  size_t off = 0;
  h.traces = off;
  off += align256(static_cast<size_t>(geo.B) * geo.M * w.pitch * 4);
  h.ants = off;
  off += align256(static_cast<size_t>(ant_stride ? geo.B : 1) * geo.M * 3 * 4);
  h.results = off;
  off += align256(static_cast<size_t>(geo.B) * sizeof(uwb_result));
  h.local = off;
  off += ws_layout(geo.B, decimate(geo.g, rule).Pd).total;
  h.total = off;
  return h;
}

int host_checks(int batch, const float* traces, int M, int N, const float* ant,
                long long ant_stride, const uwb_grid* grid, double v, double fs, int window,
                int beamformer, const uwb_rule* rule, Geo* geo) {
  int st = check_common(batch, traces, M, N, ant, grid, v, fs, window, geo);
  if (st) return st;
  if ((st = check_rule(rule))) return st;
  if (ant_stride < 0 || (ant_stride != 0 && ant_stride < 3LL * M))
    return fail(UWB_ERR_ARG, "antenna stride must be 0 or >= 3 M");
  if (bf_of(beamformer) < 0) return fail(UWB_ERR_ARG, "unknown beamformer %d", beamformer);
  return UWB_OK;
}

// ---- ragged batches: plans of per-scan descriptors --------------------------

struct PlanLayout {
  size_t descs, maps, pboxes, pprefix, fboxes, fprefix, sel, fin;  // written at upload
  size_t keys, status, counters, profiles, rboxes, rprefix;         // scratch of a run
  size_t total;
};

}  // namespace
}  // namespace uwb

// The plan of a ragged batch (host object; see uwb_plan_create).
struct uwb_plan {
  int B = 0, dtype = 0, W = 0, bf = 0, dim = 0;
  uwb_rule rule{};
  uwb::Variant var{};
  int span = 0;
  int wdim_full[3] = {32, 1, 1}, wdim_dec[3] = {32, 1, 1};
  std::vector<uwb::ScanDesc> descs;
  std::vector<CUtensorMap> maps;
  std::vector<uwb::LatBox> pboxes, fboxes;
  std::vector<int> pprefix, fprefix;
  std::vector<uwb::SelScan> sel;
  std::vector<uwb::FinScan> fin;
  std::vector<long long> img_off;
  long long img_total = 0, prof_total = 0;
  int any_tma = 0, max_iters_any = 0;
  uwb::PlanLayout lay{};
  char* ws = nullptr;  // uploaded workspace
  size_t ws_bytes = 0;
};

namespace uwb {
namespace {

PlanLayout plan_layout(const uwb_plan& pl) {
  PlanLayout L;
  const size_t B = pl.B;
  size_t off = 0;
  auto take = [&off](size_t bytes, size_t align) {
    off = align_up(off, align);
    const size_t at = off;
    off += bytes;
    return at;
  };
  L.descs = take(B * sizeof(ScanDesc), 256);
  L.maps = take(B * sizeof(CUtensorMap), 128);
  L.pboxes = take(B * sizeof(LatBox), 256);
  L.pprefix = take((B + 1) * 4, 256);
  L.fboxes = take(B * sizeof(LatBox), 256);
  L.fprefix = take((B + 1) * 4, 256);
  L.sel = take(B * sizeof(SelScan), 256);
  L.fin = take(B * sizeof(FinScan), 256);
  L.keys = take(B * 8 + 4 + 4 * kWsCounters, 256);  // keys, the status word, tile counters
  L.status = L.keys + B * 8;
  L.counters = L.status + 4;
  L.profiles = take(static_cast<size_t>(pl.prof_total) * 4, 256);
  L.rboxes = take(B * sizeof(LatBox), 256);
  L.rprefix = take((B + 1) * 4, 256);
  L.total = align_up(off, 256);
  return L;
}

ImgParams plan_params(const uwb_plan& pl, int* status) {
  ImgParams p;
  memset(&p, 0, sizeof p);
  p.B = pl.B;
  p.W = pl.W;
  p.h = pl.W / 2;
  p.span = pl.span;
  p.wpad = pl.var.wpad;
  p.dtype = pl.dtype;
  p.Mcap = pl.var.M;
  p.Rcap = pl.var.R;
  for (int a = 0; a < 3; ++a) p.tdim[a] = pl.var.tdim[a];
  p.descs = reinterpret_cast<const ScanDesc*>(pl.ws + pl.lay.descs);
  p.tmaps = pl.any_tma ? reinterpret_cast<const CUtensorMap*>(pl.ws + pl.lay.maps) : nullptr;
  p.status = status;
  p.uni.tiles = 1;
  return p;
}

int plan_launch(const uwb_plan& pl, ImgParams& p, long long work_bound, const int wdim[3],
                cudaStream_t cs, int* own_ctr) {
  Device* dev;
  int st = device(&dev);
  if (st) return st;
  for (int a = 0; a < 3; ++a) p.wdim[a] = wdim[a];
  const size_t smem =
      image_smem_layout(pl.var.bf, p.Mcap, p.Rcap, pl.var.rows, p.span, var_points(pl.var), false,
                        p.dtype)
          .total;
  const int occ = occupancy(pl.var, smem);
  if (occ < 1)
    return fail(UWB_ERR_UNSUPPORTED, "image kernel cannot launch with %zu B of shared memory", smem);
  long long ctas = static_cast<long long>(dev->sms) * occ;
  if (work_bound < ctas) ctas = work_bound;
  if (ctas < 1) return UWB_OK;
  CUtensorMap dummy;
  memset(&dummy, 0, sizeof dummy);
  cudaError_t e = launch_balanced(*dev, pl.var, p, &dummy, static_cast<int>(ctas), occ, smem,
                                  work_bound, cs, own_ctr);
  if (e != cudaSuccess) return cuda_fail(e, "image kernel launch");
  return UWB_OK;
}

}  // namespace
}  // namespace uwb

using namespace uwb;

extern "C" {

int uwb_default_rule(uwb_rule* rule) {
  if (!rule) return fail(UWB_ERR_ARG, "null rule");
  rule->mode = UWB_DECIM_AUTO;
  rule->decimation = 1;
  rule->min_tumor_diameter = 0.01;
  rule->metric = UWB_METRIC_HYBRID;
  rule->min_segment = 4;
  rule->frame_num = 1;
  rule->frame_den = 4;
  rule->max_iters = 0;
  return UWB_OK;
}

int uwb_decimation(const uwb_grid* grid, const uwb_rule* rule) {
  Geo geo;
  const float dummy = 0.f;
  int st = check_common(1, &dummy, 1, 1, &dummy, grid, 1.0, 1.0, 1, &geo);
  if (st) return st;
  if ((st = check_rule(rule))) return st;
  return decimation_of(geo.g, *rule);
}

int uwb_das_image(const float* traces, int M, int N, const float* antennas, const uwb_grid* grid,
                  double v, double fs, int window, float* image, long long* peak_index,
                  void* stream) {
  return image_impl(1, UWB_DAS, traces, M, N, antennas, 0, grid, v, fs, window, image,
                    peak_index, stream);
}

int uwb_dmas_image(const float* traces, int M, int N, const float* antennas,
                   const uwb_grid* grid, double v, double fs, int window, int literal_pairs,
                   float* image, long long* peak_index, void* stream) {
  return image_impl(1, literal_pairs ? UWB_DMAS_LITERAL : UWB_DMAS, traces, M, N, antennas, 0,
                    grid, v, fs, window, image, peak_index, stream);
}

int uwb_image_batch(int batch, int beamformer, const float* traces, int M, int N,
                    const float* antennas, long long antenna_stride, const uwb_grid* grid,
                    double v, double fs, int window, float* image, long long* peak_index,
                    void* stream) {
  return image_impl(batch, beamformer, traces, M, N, antennas, antenna_stride, grid, v, fs,
                    window, image, peak_index, stream);
}

int uwb_image_multistatic_batch(int batch, int beamformer, const float* traces, int C, int N,
                                const int* channels, const float* antennas, int M,
                                long long antenna_stride, const uwb_grid* grid, double v,
                                double fs, int window, float* image, long long* peak_index,
                                void* stream) {
  return image_impl(batch, beamformer, traces, M, N, antennas, antenna_stride, grid, v, fs,
                    window, image, peak_index, stream, C, channels);
}

size_t uwb_localize_multistatic_workspace(int batch, int C, int N, const uwb_grid* grid,
                                          int beamformer, const uwb_rule* rule) {
  if (C < 1) return 0;
  return uwb_localize_workspace(batch, 1, N, grid, beamformer, rule);
}

int uwb_localize_multistatic_batch(int batch, const float* traces, int C, int N,
                                   const int* channels, const float* antennas, int M,
                                   long long antenna_stride, const uwb_grid* grid, double v,
                                   double fs, int window, int beamformer, const uwb_rule* rule,
                                   void* workspace, size_t ws_bytes, uwb_result* out,
                                   float* image, void* stream) {
  return localize_impl(batch, traces, M, N, antennas, antenna_stride, grid, v, fs, window,
                       beamformer, rule, workspace, ws_bytes, out, image, stream, C, channels);
}

size_t uwb_localize_workspace(int batch, int M, int N, const uwb_grid* grid, int beamformer,
                              const uwb_rule* rule) {
  Geo geo;
  const float dummy = 0.f;
  if (check_common(batch, &dummy, M, N, &dummy, grid, 1.0, 1.0, 1, &geo)) return 0;
  if (check_rule(rule) || bf_of(beamformer) < 0) return 0;
  return ws_layout(batch, decimate(geo.g, *rule).Pd).total;
}

size_t uwb_presence_workspace(int batch, int M, int N, const uwb_grid* grid, int beamformer,
                              const uwb_rule* rule, int decimation2) {
  if (decimation2 < 1 || !rule) return 0;
  uwb_rule r2 = *rule;
  r2.mode = UWB_DECIM_MANUAL;
  r2.decimation = decimation2;
  const size_t a = uwb_localize_workspace(batch, M, N, grid, beamformer, rule);
  const size_t b = uwb_localize_workspace(batch, M, N, grid, beamformer, &r2);
  if (!a || !b) return 0;
  return a > b ? a : b;
}

int uwb_presence_batch(int batch, const float* traces, int M, int N, const float* antennas,
                       long long antenna_stride, const uwb_grid* grid, double v, double fs,
                       int window, int beamformer, const uwb_rule* rule, int decimation2,
                       void* workspace, size_t ws_bytes, uwb_result* out1, uwb_result* out2,
                       int* present, void* stream) {
  if (decimation2 < 1) return fail(UWB_ERR_ARG, "second decimation factor %d < 1", decimation2);
  if (!out2 || !present) return fail(UWB_ERR_ARG, "null second result array or verdicts");
  int st = localize_impl(batch, traces, M, N, antennas, antenna_stride, grid, v, fs, window,
                         beamformer, rule, workspace, ws_bytes, out1, nullptr, stream);
  if (st) return st;
  uwb_rule r2 = *rule;
  r2.mode = UWB_DECIM_MANUAL;
  r2.decimation = decimation2;
  st = localize_impl(batch, traces, M, N, antennas, antenna_stride, grid, v, fs, window,
                     beamformer, &r2, workspace, ws_bytes, out2, nullptr, stream);
  if (st) return st;
  cudaError_t e = launch_presence(out1, out2, present, batch, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "presence launch");
  return UWB_OK;
}

size_t uwb_localize_host_workspace(int batch, const float* traces_host, int M, int N,
                                   const float* antennas_host, long long antenna_stride,
                                   const uwb_grid* grid, double v, double fs, int window,
                                   int beamformer, const uwb_rule* rule) {
  Geo geo;
  if (host_checks(batch, traces_host, M, N, antennas_host, antenna_stride, grid, v, fs, window,
                  beamformer, rule, &geo))
    return 0;
  const HostWindow w = reachable_window(geo, antennas_host, antenna_stride);
  return host_layout(geo, w, antenna_stride, *rule).total;
}

int uwb_localize_host(int batch, const float* traces_host, int M, int N,
                      const float* antennas_host, long long antenna_stride, const uwb_grid* grid,
                      double v, double fs, int window, int beamformer, const uwb_rule* rule,
                      void* workspace, size_t ws_bytes, uwb_result* out_host,
                      long long* h2d_bytes, void* stream) {
  Geo geo;
  int st = host_checks(batch, traces_host, M, N, antennas_host, antenna_stride, grid, v, fs,
                       window, beamformer, rule, &geo);
  if (st) return st;
  if (!out_host) return fail(UWB_ERR_ARG, "null result array");
  const HostWindow w = reachable_window(geo, antennas_host, antenna_stride);
  const HostLayout hl = host_layout(geo, w, antenna_stride, *rule);
  if (!workspace) return fail(UWB_ERR_WORKSPACE, "null workspace");
  if (reinterpret_cast<uintptr_t>(workspace) & 255)
    return fail(UWB_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (ws_bytes < hl.total)
    return fail(UWB_ERR_WORKSPACE, "workspace of %zu bytes < %zu needed", ws_bytes, hl.total);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  float* dtr = reinterpret_cast<float*>(ws + hl.traces);
  float* dant = reinterpret_cast<float*>(ws + hl.ants);
  uwb_result* dres = reinterpret_cast<uwb_result*>(ws + hl.results);
  const size_t ant_bytes = static_cast<size_t>(antenna_stride ? batch : 1) * M * 3 * 4;
  long long moved = 0;
  cudaError_t e;
  if (w.len > 0) {
    e = cudaMemcpy2DAsync(dtr, static_cast<size_t>(w.pitch) * 4, traces_host + w.w0,
                          static_cast<size_t>(N) * 4, static_cast<size_t>(w.len) * 4,
                          static_cast<size_t>(batch) * M, cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return cuda_fail(e, "trace window copy");
    moved += static_cast<long long>(batch) * M * w.len * 4;
  }
  if (antenna_stride) {
    // pack the per-scan arrays densely on the device
    e = cudaMemcpy2DAsync(dant, static_cast<size_t>(M) * 12, antennas_host,
                          static_cast<size_t>(antenna_stride) * 4, static_cast<size_t>(M) * 12,
                          static_cast<size_t>(batch), cudaMemcpyHostToDevice, cs);
  } else {
    e = cudaMemcpyAsync(dant, antennas_host, ant_bytes, cudaMemcpyHostToDevice, cs);
  }
  if (e != cudaSuccess) return cuda_fail(e, "antenna copy");
  moved += static_cast<long long>(ant_bytes);
  Geo dgeo = geo;
  dgeo.N = w.len;
  dgeo.pitch = w.pitch;
  dgeo.n_begin = w.w0;
  st = localize_core(dgeo, dtr, dant, antenna_stride ? 3LL * M : 0, beamformer, rule,
                     ws + hl.local, hl.total - hl.local, dres, nullptr, stream);
  if (st) return st;
  e = cudaMemcpyAsync(out_host, dres, static_cast<size_t>(batch) * sizeof(uwb_result),
                      cudaMemcpyDeviceToHost, cs);
  if (e != cudaSuccess) return cuda_fail(e, "result copy");
  if (h2d_bytes) *h2d_bytes = moved;
  return UWB_OK;
}

int uwb_localize(const float* traces, int M, int N, const float* antennas, const uwb_grid* grid,
                 double v, double fs, int window, int beamformer, const uwb_rule* rule,
                 void* workspace, size_t ws_bytes, uwb_result* out, float* image, void* stream) {
  return localize_impl(1, traces, M, N, antennas, 0, grid, v, fs, window, beamformer, rule,
                       workspace, ws_bytes, out, image, stream);
}

int uwb_localize_batch(int batch, const float* traces, int M, int N, const float* antennas,
                       long long antenna_stride, const uwb_grid* grid, double v, double fs,
                       int window, int beamformer, const uwb_rule* rule, void* workspace,
                       size_t ws_bytes, uwb_result* out, float* image, void* stream) {
  return localize_impl(batch, traces, M, N, antennas, antenna_stride, grid, v, fs, window,
                       beamformer, rule, workspace, ws_bytes, out, image, stream);
}

}  // extern "C"

// Scratch of uwb_localize_batch_noalloc: a fixed array in the library image,
// one copy per device, so callers that may not allocate still get a
// workspace. In host code `g_noalloc_scratch` only names the symbol; the
// device address comes from cudaGetSymbolAddress, looked up once per device
// with that device current.
static __device__ __align__(256) unsigned char g_noalloc_scratch[UWB_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {};

int noalloc_scratch(void** out) {
  int d = 0;
  cudaError_t e = cudaGetDevice(&d);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (d < 0 || d >= 64) return fail(UWB_ERR_UNSUPPORTED, "device ordinal %d", d);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[d]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_noalloc_ptr[d] = p;
  }
  *out = g_noalloc_ptr[d];
  return UWB_OK;
}
}  // namespace

extern "C" {

int uwb_localize_batch_noalloc(int batch, const float* traces, int M, int N,
                               const float* antennas, long long antenna_stride,
                               const uwb_grid* grid, double v, double fs, int window,
                               int beamformer, const uwb_rule* rule, uwb_result* out,
                               float* image, void* stream) {
  const size_t need = uwb_localize_workspace(batch, M, N, grid, beamformer, rule);
  if (need == 0) {
    // invalid arguments: let the regular checks name the problem
    return localize_impl(batch, traces, M, N, antennas, antenna_stride, grid, v, fs, window,
                         beamformer, rule, nullptr, 0, out, image, stream);
  }
  if (need > UWB_NOALLOC_SCRATCH_BYTES)
    return fail(UWB_ERR_WORKSPACE,
                "this call needs %zu bytes of scratch but the built-in scratch holds %u; "
                "use a smaller batch or uwb_localize_batch with a workspace",
                need, UWB_NOALLOC_SCRATCH_BYTES);
  void* scratch = nullptr;
  int st = noalloc_scratch(&scratch);
  if (st) return st;
  return localize_impl(batch, traces, M, N, antennas, antenna_stride, grid, v, fs, window,
                       beamformer, rule, scratch, UWB_NOALLOC_SCRATCH_BYTES, out, image, stream);
}

uwb_plan* uwb_plan_create(int batch, const uwb_scan* scans, int dtype, int window,
                          int beamformer, const uwb_rule* rule, int* status) {
  auto bad = [status](int code) -> uwb_plan* {
    if (status) *status = code;
    return nullptr;
  };
  if (batch < 1 || batch > (1 << 22) || !scans)
    return bad(fail(UWB_ERR_ARG, "a plan needs 1..2^22 scans"));
  if (dtype != UWB_F32 && dtype != UWB_F16 && dtype != UWB_BF16)
    return bad(fail(UWB_ERR_ARG, "unknown trace element type %d", dtype));
  int st = check_rule(rule);
  if (st) return bad(st);
  const int bf = bf_of(beamformer);
  if (bf < 0) return bad(fail(UWB_ERR_ARG, "unknown beamformer %d", beamformer));
  std::unique_ptr<uwb_plan> pl(new uwb_plan);
  pl->B = batch;
  pl->dtype = dtype;
  pl->W = window;
  pl->bf = bf;
  pl->rule = *rule;
  pl->dim = scans[0].grid.dim;
  int Mcap = 0;
  double max_delta = 0.0;
  std::vector<Geo> geos(batch);
  for (int b = 0; b < batch; ++b) {
    const uwb_scan& sc = scans[b];
    st = check_common(1, static_cast<const float*>(sc.traces), sc.M, sc.N, sc.antennas, &sc.grid,
                      sc.v, sc.fs, window, &geos[b]);
    if (st) {
      char why[sizeof t_err];
      snprintf(why, sizeof why, "%s", t_err);
      return bad(fail(st, "scan %d: %s", b, why));
    }
    if (sc.grid.dim != pl->dim) return bad(fail(UWB_ERR_ARG, "scan %d: all scans of a plan "
                                                "share the grid dimensionality", b));
    Mcap = sc.M > Mcap ? sc.M : Mcap;
    for (int a = 0; a < sc.grid.dim; ++a)
      max_delta = std::fmax(max_delta, sc.grid.pitch[a] * geos[b].kscale);
  }
  if ((st = pick_variant(bf, Mcap, window, pl->dim, &pl->var))) return bad(st);
  use_ragged_shape(&pl->var);
  pl->span = pick_span(pl->var, Mcap, dtype);
  const double d1[3] = {max_delta, max_delta, pl->dim == 3 ? max_delta : 1e9};
  pick_warp(pl->var.tdim, d1, pl->wdim_full);
  pl->descs.resize(batch);
  pl->maps.resize(batch);
  pl->pboxes.resize(batch);
  pl->fboxes.resize(batch);
  pl->sel.resize(batch);
  pl->fin.resize(batch);
  pl->img_off.resize(batch);
  pl->pprefix.assign(batch + 1, 0);
  pl->fprefix.assign(batch + 1, 0);
  double max_dec = 0.0;
  for (int b = 0; b < batch; ++b) {
    const uwb_scan& sc = scans[b];
    const Geo& g = geos[b];
    const Decim dc = decimate(g.g, *rule);
    ScanDesc& d = pl->descs[b];
    memset(&d, 0, sizeof d);
    d.traces = sc.traces;
    d.ant = sc.antennas;
    d.img_off = pl->img_total;
    d.cmp_off = pl->prof_total;
    d.pitch = sc.N;
    d.n_begin = 0;
    d.N = sc.N;
    d.M = sc.M;
    d.R = sc.M;
    d.kscale = g.kscale;
    for (int a = 0; a < 3; ++a) {
      d.org[a] = static_cast<float>(g.g.origin[a]);
      d.pit[a] = static_cast<float>(g.g.pitch[a]);
      d.gn[a] = g.g.n[a];
    }
    d.tma = encode_map(sc.traces, dtype, sc.N, sc.N, 0, sc.M, 1, pl->span, &pl->maps[b]) ? b : -1;
    pl->any_tma |= d.tma >= 0;
    pl->img_off[b] = pl->img_total;
    pl->img_total += g.P;
    LatBox& pb = pl->pboxes[b];
    LatBox& fb = pl->fboxes[b];
    for (int a = 0; a < 3; ++a) {
      pb.lo[a] = dc.off[a];
      pb.step[a] = dc.step[a];
      pb.cnt[a] = dc.cnt[a];
      fb.lo[a] = 0;
      fb.step[a] = 1;
      fb.cnt[a] = g.g.n[a];
      max_dec = std::fmax(max_dec, dc.step[a] * g.g.pitch[a] * g.kscale * (a < pl->dim));
    }
    pb.tiles = lattice_tiles(pb.cnt, pl->var.tdim);
    fb.tiles = lattice_tiles(fb.cnt, pl->var.tdim);
    pl->pprefix[b + 1] = pl->pprefix[b] + pb.tiles;
    pl->fprefix[b + 1] = pl->fprefix[b] + fb.tiles;
    SelScan& q = pl->sel[b];
    q.prof_off = pl->prof_total;
    for (int a = 0; a < 3; ++a) {
      q.gn[a] = g.g.n[a];
      q.off[a] = dc.off[a];
      q.step[a] = dc.step[a];
      q.cnt[a] = dc.cnt[a];
    }
    q.D = dc.D;
    q.max_iters = dc.max_iters;
    FinScan& f = pl->fin[b];
    for (int a = 0; a < 3; ++a) {
      f.gn[a] = g.g.n[a];
      f.org[a] = g.g.origin[a];
      f.pit[a] = g.g.pitch[a];
    }
    f.Pd = dc.Pd;
    pl->prof_total += dc.Pd;
  }
  const double d2[3] = {max_dec, max_dec, pl->dim == 3 ? max_dec : 1e9};
  pick_warp(pl->var.tdim, d2, pl->wdim_dec);
  pl->lay = plan_layout(*pl);
  if (status) *status = UWB_OK;
  return pl.release();
}

size_t uwb_plan_workspace(const uwb_plan* plan) { return plan ? plan->lay.total : 0; }

long long uwb_plan_image_offset(const uwb_plan* plan, int scan) {
  if (!plan || scan < 0 || scan > plan->B) return -1;
  return scan == plan->B ? plan->img_total : plan->img_off[scan];
}

int uwb_plan_upload(uwb_plan* plan, void* workspace, size_t ws_bytes, void* stream) {
  if (!plan) return fail(UWB_ERR_ARG, "null plan");
  if (!workspace) return fail(UWB_ERR_WORKSPACE, "null workspace");
  if (reinterpret_cast<uintptr_t>(workspace) & 255)
    return fail(UWB_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (ws_bytes < plan->lay.total)
    return fail(UWB_ERR_WORKSPACE, "workspace of %zu bytes < %zu needed", ws_bytes,
                plan->lay.total);
  Device* dev;
  int st = device(&dev);
  if (st) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  const size_t B = plan->B;
  struct {
    size_t at;
    const void* src;
    size_t bytes;
  } parts[] = {
      {plan->lay.descs, plan->descs.data(), B * sizeof(ScanDesc)},
      {plan->lay.maps, plan->maps.data(), B * sizeof(CUtensorMap)},
      {plan->lay.pboxes, plan->pboxes.data(), B * sizeof(LatBox)},
      {plan->lay.pprefix, plan->pprefix.data(), (B + 1) * 4},
      {plan->lay.fboxes, plan->fboxes.data(), B * sizeof(LatBox)},
      {plan->lay.fprefix, plan->fprefix.data(), (B + 1) * 4},
      {plan->lay.sel, plan->sel.data(), B * sizeof(SelScan)},
      {plan->lay.fin, plan->fin.data(), B * sizeof(FinScan)},
  };
  for (const auto& part : parts) {
    cudaError_t e = cudaMemcpyAsync(ws + part.at, part.src, part.bytes, cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return cuda_fail(e, "plan upload");
  }
  plan->ws = ws;
  plan->ws_bytes = ws_bytes;
  return UWB_OK;
}

int uwb_plan_images(uwb_plan* plan, float* images, long long* peak_index, void* stream) {
  if (!plan || !plan->ws) return fail(UWB_ERR_ARG, "plan not uploaded");
  if (!images) return fail(UWB_ERR_ARG, "null images");
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  int* status = reinterpret_cast<int*>(plan->ws + plan->lay.status);
  int* counters = reinterpret_cast<int*>(plan->ws + plan->lay.counters);
  // the status word and the tile counters start at zero
  cudaError_t e = cudaMemsetAsync(status, 0, 4 + 4 * kWsCounters, cs);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  if (peak_index) {
    e = cudaMemsetAsync(peak_index, 0, sizeof(long long) * plan->B, cs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  }
  ImgParams p = plan_params(*plan, status);
  p.boxes = reinterpret_cast<const LatBox*>(plan->ws + plan->lay.fboxes);
  p.prefix = reinterpret_cast<const int*>(plan->ws + plan->lay.fprefix);
  p.image = images;
  p.keys = reinterpret_cast<unsigned long long*>(peak_index);
  int st = plan_launch(*plan, p, plan->fprefix[plan->B], plan->wdim_full, cs, counters);
  if (st) return st;
  if (peak_index) {
    e = launch_keys_to_index(p.keys, plan->B, cs);
    if (e != cudaSuccess) return cuda_fail(e, "argmax decode launch");
  }
  return UWB_OK;
}

int uwb_plan_localize(uwb_plan* plan, uwb_result* out, void* stream) {
  if (!plan || !plan->ws) return fail(UWB_ERR_ARG, "plan not uploaded");
  if (!out) return fail(UWB_ERR_ARG, "null result array");
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  char* ws = plan->ws;
  const PlanLayout& L = plan->lay;
  const int B = plan->B;
  int* status = reinterpret_cast<int*>(ws + L.status);
  auto* keys = reinterpret_cast<unsigned long long*>(ws + L.keys);
  auto* rboxes = reinterpret_cast<LatBox*>(ws + L.rboxes);
  auto* rprefix = reinterpret_cast<int*>(ws + L.rprefix);
  int* counters = reinterpret_cast<int*>(ws + L.counters);
  // keys, status word and tile counters start at zero
  cudaError_t e =
      cudaMemsetAsync(ws + L.keys, 0, static_cast<size_t>(B) * 8 + 4 + 4 * kWsCounters, cs);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  PhaseTimer timer(cs);
  timer.mark();
  // 1. decimated profiles
  ImgParams p1 = plan_params(*plan, status);
  p1.boxes = reinterpret_cast<const LatBox*>(ws + L.pboxes);
  p1.prefix = reinterpret_cast<const int*>(ws + L.pprefix);
  p1.compact = reinterpret_cast<float*>(ws + L.profiles);
  int st = plan_launch(*plan, p1, plan->pprefix[B], plan->wdim_dec, cs, counters);
  if (st) return st;
  timer.mark();
  // 2. selection (per-scan lattices) and work planning
  SelParams sp;
  memset(&sp, 0, sizeof sp);
  sp.scans = reinterpret_cast<const SelScan*>(ws + L.sel);
  sp.profile = reinterpret_cast<const float*>(ws + L.profiles);
  sp.B = B;
  sp.dim = plan->dim;
  for (int a = 0; a < 3; ++a) sp.tdim[a] = plan->var.tdim[a];
  sp.rule = plan->rule;
  sp.boxes = rboxes;
  sp.out = out;
  if ((e = launch_select(sp, cs)) != cudaSuccess) return cuda_fail(e, "select launch");
  if ((e = launch_plan(rboxes, rprefix, B, cs)) != cudaSuccess) return cuda_fail(e, "plan launch");
  timer.mark();
  // 3. final regions at full resolution + argmax
  ImgParams p2 = plan_params(*plan, status);
  p2.boxes = rboxes;
  p2.prefix = rprefix;
  p2.keys = keys;
  if ((st = plan_launch(*plan, p2, plan->fprefix[B], plan->wdim_full, cs, counters + 1)))
    return st;
  timer.mark();
  FinishParams fp;
  memset(&fp, 0, sizeof fp);
  fp.scans = reinterpret_cast<const FinScan*>(ws + L.fin);
  fp.keys = keys;
  fp.boxes = rboxes;
  fp.out = out;
  fp.B = B;
  if ((e = launch_finish(fp, status, cs)) != cudaSuccess) return cuda_fail(e, "finish launch");
  timer.mark();
  timer.commit();
  return UWB_OK;
}

void uwb_plan_destroy(uwb_plan* plan) { delete plan; }

int uwb_tile_shape(int beamformer, int dim, int tile[3]) {
  const int bf = bf_of(beamformer);
  if (bf < 0 || (dim != 2 && dim != 3) || !tile) return fail(UWB_ERR_ARG, "bad tile query");
  Variant v;
  int st = pick_variant(bf, 16, 20, dim, &v);
  if (st) return st;
  for (int a = 0; a < 3; ++a) tile[a] = tile_linear(v.tdim) ? 0 : v.tdim[a];
  return UWB_OK;
}

int uwb_set_tile_shape(int beamformer, int dim, const int tile[3]) {
  const int bf = bf_of(beamformer);
  if (bf < 0 || (dim != 2 && dim != 3)) return fail(UWB_ERR_ARG, "bad beamformer or dim");
  std::lock_guard<std::mutex> lk(g_tile_mu);
  if (!tile) {
    for (int a = 0; a < 3; ++a) g_tile[bf][dim][a] = 0;
    return UWB_OK;
  }
  const bool linear = tile[0] == 0 && tile[1] == 0 && tile[2] == 0;
  if (!tile_ok(bf, tile) || (dim == 2 && tile[2] != 1 && !linear))
    return fail(UWB_ERR_ARG,
                "tile must be {0, 0, 0} (linear) or powers of two multiplying to the CTA size");
  for (int a = 0; a < 3; ++a) g_tile[bf][dim][a] = tile[a];
  return UWB_OK;
}

int uwb_autotune(int batch, const uwb_scan* scans, int dtype, int window, int beamformer,
                 const uwb_rule* rule, void* workspace, size_t ws_bytes, uwb_result* out,
                 int tile_out[3], float* ms_out, void* stream) {
  const int bf = bf_of(beamformer);
  if (bf < 0 || !scans || batch < 1) return fail(UWB_ERR_ARG, "bad autotune arguments");
  const int dim = scans[0].grid.dim;
  if (dim != 2 && dim != 3) return fail(UWB_ERR_ARG, "grid dim must be 2 or 3");
  // linear tiles ({0, 0, 0}) and four shaped ones
  static const int c256_2[][3] = {{0, 0, 0}, {32, 8, 1}, {16, 16, 1}, {64, 4, 1}, {8, 32, 1}};
  static const int c128_2[][3] = {{0, 0, 0}, {16, 8, 1}, {32, 4, 1}, {8, 16, 1}, {64, 2, 1}};
  static const int c256_3[][3] = {{0, 0, 0}, {16, 4, 4}, {8, 8, 4}, {32, 4, 2}, {8, 4, 8}};
  static const int c128_3[][3] = {{0, 0, 0}, {8, 4, 4}, {16, 4, 2}, {4, 8, 4}, {8, 8, 2}};
  const int n_cand = 5;
  const int(*cand)[3] = bf == BF_DMAS_LIT ? (dim == 2 ? c128_2 : c128_3)
                                          : (dim == 2 ? c256_2 : c256_3);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(UWB_ERR_CUDA, "cudaEventCreate");
  float best_ms = 1e30f;
  int best = -1, st = UWB_OK;
  int saved[3];
  {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    for (int a = 0; a < 3; ++a) saved[a] = g_tile[bf][dim][a];
  }
  for (int c = 0; c < n_cand && st == UWB_OK; ++c) {
    st = uwb_set_tile_shape(beamformer, dim, cand[c]);
    if (st) break;
    uwb_plan* plan = uwb_plan_create(batch, scans, dtype, window, beamformer, rule, &st);
    if (!plan) break;
    if ((st = uwb_plan_upload(plan, workspace, ws_bytes, stream)) == UWB_OK &&
        (st = uwb_plan_localize(plan, out, stream)) == UWB_OK) {  // warm-up
      cudaEventRecord(e0, cs);
      st = uwb_plan_localize(plan, out, stream);
      cudaEventRecord(e1, cs);
      if (st == UWB_OK && cudaEventSynchronize(e1) == cudaSuccess) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
          best_ms = ms;
          best = c;
        }
      }
    }
    uwb_plan_destroy(plan);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_tile_mu);
  if (st != UWB_OK || best < 0) {
    for (int a = 0; a < 3; ++a) g_tile[bf][dim][a] = saved[a];
    return st ? st : fail(UWB_ERR_CUDA, "autotune timed nothing");
  }
  for (int a = 0; a < 3; ++a) {
    g_tile[bf][dim][a] = cand[best][a];
    if (tile_out) tile_out[a] = cand[best][a];
  }
  if (ms_out) *ms_out = best_ms;
  return UWB_OK;
}

int uwb_phase_timing(int enable) {
  std::lock_guard<std::mutex> lk(g_timing_mu);
  drop_records();
  g_timing = enable != 0;
  return UWB_OK;
}

int uwb_phase_times(double* ms) {
  if (!ms) return fail(UWB_ERR_ARG, "null ms");
  std::lock_guard<std::mutex> lk(g_timing_mu);
  for (int p = 0; p < kPhases; ++p) ms[p] = 0.0;
  const int calls = static_cast<int>(g_phase_records.size());
  for (auto& r : g_phase_records) {
    cudaError_t e = cudaEventSynchronize(r.ev[kPhases]);
    if (e != cudaSuccess) {
      drop_records();
      return cuda_fail(e, "cudaEventSynchronize");
    }
    for (int p = 0; p < kPhases; ++p) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, r.ev[p], r.ev[p + 1]);
      if (e != cudaSuccess) {
        drop_records();
        return cuda_fail(e, "cudaEventElapsedTime");
      }
      ms[p] += t;
    }
  }
  drop_records();
  return calls;
}

int uwb_device_status(int clear) {
  Device* dev;
  int st = device(&dev);
  if (st) return st;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  int word = 0;
  e = cudaMemcpy(&word, dev->status, sizeof word, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
  if (clear) {
    e = cudaMemset(dev->status, 0, sizeof word);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
  }
  return word;
}

const char* uwb_last_error(void) { return t_err; }

}  // extern "C"

// ---------------------------------------------------- learned segment proposal
namespace {

// The tensor-core self-check, once per device: an integer-valued BF16 GEMM
// through the network's descriptor, TMEM and epilogue conventions, compared
// exactly on the host. The network's kernels only run where it passed.
std::mutex g_umma_mu;
int g_umma_state[64] = {};  // 0 unknown, 1 passed, -1 failed

uint16_t bf16_bits_of_small_int(int v) {
  const float f = static_cast<float>(v);
  uint32_t u;
  memcpy(&u, &f, 4);
  return static_cast<uint16_t>(u >> 16);  // exact for small integers
}

int umma_selftest_run(int* passed) {
  Device* dev;
  int st = device(&dev);
  if (st) return st;
  int d = 0;
  cudaError_t e = cudaGetDevice(&d);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_umma_mu);
  if (g_umma_state[d] != 0) {
    *passed = g_umma_state[d] > 0;
    return UWB_OK;
  }
  std::vector<uint16_t> A(128 * 64), B(32 * 64);
  std::vector<int> Ai(128 * 64), Bi(32 * 64);
  for (int m = 0; m < 128; ++m)
    for (int k = 0; k < 64; ++k) {
      Ai[m * 64 + k] = (m * 7 + k * 3) % 9 - 4;
      A[m * 64 + k] = bf16_bits_of_small_int(Ai[m * 64 + k]);
    }
  for (int n = 0; n < 32; ++n)
    for (int k = 0; k < 64; ++k) {
      Bi[n * 64 + k] = (n * 5 + k * 11 + 1) % 9 - 4;
      B[n * 64 + k] = bf16_bits_of_small_int(Bi[n * 64 + k]);
    }
  void *dA = nullptr, *dB = nullptr, *dD = nullptr, *dS = nullptr;
  std::vector<float> D(128 * 32, 0.f);
  int sw = 0;
  cudaStream_t cs = nullptr;
  auto cleanup = [&]() {
    if (cs) cudaStreamDestroy(cs);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD);
    cudaFree(dS);
  };
  if ((e = cudaMalloc(&dA, A.size() * 2)) != cudaSuccess ||
      (e = cudaMalloc(&dB, B.size() * 2)) != cudaSuccess ||
      (e = cudaMalloc(&dD, D.size() * 4)) != cudaSuccess ||
      (e = cudaMalloc(&dS, 4)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dA, A.data(), A.size() * 2, cudaMemcpyHostToDevice, cs)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dB, B.data(), B.size() * 2, cudaMemcpyHostToDevice, cs)) != cudaSuccess ||
      (e = cudaMemsetAsync(dD, 0, D.size() * 4, cs)) != cudaSuccess ||
      (e = cudaMemsetAsync(dS, 0, 4, cs)) != cudaSuccess ||
      (e = cnn::launch_selftest(static_cast<uint16_t*>(dA), static_cast<uint16_t*>(dB),
                                static_cast<float*>(dD), static_cast<int*>(dS), cs)) != cudaSuccess ||
      (e = cudaMemcpyAsync(D.data(), dD, D.size() * 4, cudaMemcpyDeviceToHost, cs)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&sw, dS, 4, cudaMemcpyDeviceToHost, cs)) != cudaSuccess ||
      (e = cudaStreamSynchronize(cs)) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "tensor-core self-check");
  }
  cleanup();
  bool ok = sw == UWB_OK;
  for (int m = 0; m < 128 && ok; ++m)
    for (int n = 0; n < 32 && ok; ++n) {
      int ref = 0;
      for (int k = 0; k < 64; ++k) ref += Ai[m * 64 + k] * Bi[n * 64 + k];
      ok = D[m * 32 + n] == static_cast<float>(ref);
    }
  g_umma_state[d] = ok ? 1 : -1;
  *passed = ok;
  return UWB_OK;
}

int umma_ready() {
  int passed = 0;
  int st = umma_selftest_run(&passed);
  if (st) return st;
  if (!passed)
    return fail(UWB_ERR_UNSUPPORTED,
                "tensor-core self-check failed on this device: the network's kernels are disabled");
  return UWB_OK;
}

int cnn_ctas(const Device& dev, int batch) { return batch < dev.sms ? batch : dev.sms; }

size_t train_layout_grad(int batch) { return align256(static_cast<size_t>(batch) * cnn::SAVE_BYTES); }

int check_cnn_batch(int batch) {
  if (batch < 1 || batch > (1 << 20)) return fail(UWB_ERR_ARG, "batch %d out of range", batch);
  return UWB_OK;
}

int cnn_gradients_impl(const void* packed, const float* maps, const int* labels, int batch,
                       float* grad, float* loss, void* ws, size_t ws_bytes, cudaStream_t cs) {
  int st;
  if ((st = check_cnn_batch(batch))) return st;
  if (!packed || !maps || !labels || !grad || !loss) return fail(UWB_ERR_ARG, "null argument");
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255))
    return fail(UWB_ERR_WORKSPACE, "workspace must be non-null and 256-byte aligned");
  if (ws_bytes < static_cast<size_t>(batch) * cnn::SAVE_BYTES)
    return fail(UWB_ERR_WORKSPACE, "workspace of %zu bytes < %zu needed", ws_bytes,
                static_cast<size_t>(batch) * cnn::SAVE_BYTES);
  if ((st = umma_ready())) return st;
  Device* dev;
  if ((st = device(&dev))) return st;
  cudaError_t e;
  if ((e = cudaMemsetAsync(grad, 0, cnn::N_PARAMS * 4, cs)) != cudaSuccess ||
      (e = cudaMemsetAsync(loss, 0, 4, cs)) != cudaSuccess)
    return cuda_fail(e, "cudaMemsetAsync");
  const int ctas = cnn_ctas(*dev, batch);
  if ((e = cnn::launch_forward(packed, maps, batch, nullptr, labels, ws, loss, dev->status, ctas,
                               cs)) != cudaSuccess)
    return cuda_fail(e, "network forward launch");
  if ((e = cnn::launch_backward(packed, ws, batch, grad, ctas, cs)) != cudaSuccess)
    return cuda_fail(e, "network backward launch");
  return UWB_OK;
}

}  // namespace

extern "C" {

int uwb_cnn_selftest(int* passed) {
  if (!passed) return fail(UWB_ERR_ARG, "null passed");
  return umma_selftest_run(passed);
}

int uwb_cnn_pack(const float* theta, void* packed, void* stream) {
  if (!theta || !packed) return fail(UWB_ERR_ARG, "null theta or packed");
  cudaError_t e = cnn::launch_pack(theta, packed, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? UWB_OK : cuda_fail(e, "pack launch");
}

int uwb_cnn_forward(const void* packed, const float* maps, int batch, float* scores,
                    void* stream) {
  int st;
  if ((st = check_cnn_batch(batch))) return st;
  if (!packed || !maps || !scores) return fail(UWB_ERR_ARG, "null argument");
  if ((st = umma_ready())) return st;
  Device* dev;
  if ((st = device(&dev))) return st;
  cudaError_t e = cnn::launch_forward(packed, maps, batch, scores, nullptr, nullptr, nullptr,
                                      dev->status, cnn_ctas(*dev, batch),
                                      static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? UWB_OK : cuda_fail(e, "network forward launch");
}

static_assert(cnn::SAVE_BYTES == UWB_CNN_RECORD_BYTES && cnn::SAVE_A1 == 5120 &&
                  cnn::SAVE_A2 == 83584 && cnn::SAVE_A3 == 162048 && cnn::SAVE_F == 240512 &&
                  cnn::SAVE_DZ == 242560 && cnn::LBO_ACT == 19616 && cnn::PAD0 == 34 &&
                  cnn::Q == 33,
              "the record layout documented in uwb.h");

int uwb_cnn_forward_record(const void* packed, const float* maps, const int* labels, int batch,
                           float* scores, float* loss, void* record, size_t record_bytes,
                           void* stream) {
  int st;
  if ((st = check_cnn_batch(batch))) return st;
  if (!packed || !maps || !scores) return fail(UWB_ERR_ARG, "null argument");
  if (labels && !loss) return fail(UWB_ERR_ARG, "labels need a loss");
  if (!record || (reinterpret_cast<uintptr_t>(record) & 255))
    return fail(UWB_ERR_WORKSPACE, "record must be non-null and 256-byte aligned");
  if (record_bytes < static_cast<size_t>(batch) * cnn::SAVE_BYTES)
    return fail(UWB_ERR_WORKSPACE, "record of %zu bytes < %zu needed", record_bytes,
                static_cast<size_t>(batch) * cnn::SAVE_BYTES);
  if ((st = umma_ready())) return st;
  Device* dev;
  if ((st = device(&dev))) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (labels && (e = cudaMemsetAsync(loss, 0, 4, cs)) != cudaSuccess)
    return cuda_fail(e, "cudaMemsetAsync");
  e = cnn::launch_forward(packed, maps, batch, scores, labels, record, labels ? loss : nullptr,
                          dev->status, cnn_ctas(*dev, batch), cs);
  return e == cudaSuccess ? UWB_OK : cuda_fail(e, "network forward launch");
}

size_t uwb_cnn_train_workspace(int batch) {
  if (batch < 1 || batch > (1 << 20)) return 0;
  return train_layout_grad(batch) + align256(cnn::N_PARAMS * 4);
}

int uwb_cnn_gradients(const void* packed, const float* maps, const int* labels, int batch,
                      float* grad, float* loss, void* workspace, size_t ws_bytes, void* stream) {
  return cnn_gradients_impl(packed, maps, labels, batch, grad, loss, workspace, ws_bytes,
                            static_cast<cudaStream_t>(stream));
}

int uwb_cnn_adam(float* theta, float* m, float* v, float* grad, void* packed, int step, float lr,
                 void* stream) {
  if (!theta || !m || !v || !grad || !packed) return fail(UWB_ERR_ARG, "null argument");
  if (step < 1) return fail(UWB_ERR_ARG, "Adam step counts from 1 (got %d)", step);
  if (!(lr > 0.f)) return fail(UWB_ERR_ARG, "learning rate must be positive");
  const double b1 = 0.9, b2 = 0.999;
  cnn::AdamConsts k;
  k.lr = lr;
  k.beta1 = static_cast<float>(b1);
  k.beta2 = static_cast<float>(b2);
  k.one_minus_beta1 = static_cast<float>(1.0 - b1);
  k.one_minus_beta2 = static_cast<float>(1.0 - b2);
  k.eps = 1e-8f;
  k.c1 = static_cast<float>(1.0 / (1.0 - std::pow(b1, step)));
  k.c2 = static_cast<float>(1.0 / (1.0 - std::pow(b2, step)));
  cudaError_t e = cnn::launch_adam(theta, m, v, grad, packed, k, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? UWB_OK : cuda_fail(e, "Adam launch");
}

int uwb_cnn_train_step(float* theta, float* m, float* v, void* packed, const float* maps,
                       const int* labels, int batch, int step, float lr, float* loss,
                       void* workspace, size_t ws_bytes, void* stream) {
  const size_t need = uwb_cnn_train_workspace(batch);
  if (need == 0) return fail(UWB_ERR_ARG, "batch %d out of range", batch);
  if (ws_bytes < need)
    return fail(UWB_ERR_WORKSPACE, "workspace of %zu bytes < %zu needed", ws_bytes, need);
  if (!workspace) return fail(UWB_ERR_WORKSPACE, "null workspace");
  float* grad = reinterpret_cast<float*>(static_cast<char*>(workspace) + train_layout_grad(batch));
  int st = cnn_gradients_impl(packed, maps, labels, batch, grad, loss, workspace,
                              train_layout_grad(batch), static_cast<cudaStream_t>(stream));
  if (st) return st;
  return uwb_cnn_adam(theta, m, v, grad, packed, step, lr, stream);
}

}  // extern "C"

// ---- coarse DAS maps and the learned localisation
namespace {

struct LearnLayout {
  size_t keys, status, maps, scores, state, map_boxes, final_boxes, prof_boxes, learned, prefix,
      profile, total;
};

LearnLayout learn_layout(int B, long long Pd) {
  LearnLayout w;
  size_t off = 0;
  w.keys = off;
  off += static_cast<size_t>(B) * 8;
  w.status = off;
  off = align256(off + 4);
  w.maps = off;
  off += align256(static_cast<size_t>(B) * cnn::MAP * cnn::MAP * 4);
  w.scores = off;
  off += align256(static_cast<size_t>(B) * cnn::SEGS * 4);
  w.state = off;
  off += align256(static_cast<size_t>(B) * sizeof(LearnState));
  w.map_boxes = off;
  off += align256(static_cast<size_t>(B) * sizeof(LatBox));
  w.final_boxes = off;
  off += align256(static_cast<size_t>(B) * sizeof(LatBox));
  w.prof_boxes = off;
  off += align256(static_cast<size_t>(B) * sizeof(LatBox));
  w.learned = off;
  off += align256(static_cast<size_t>(B) * 4);
  w.prefix = off;
  off += align256(static_cast<size_t>(B + 1) * 4);
  w.profile = off;
  off += align256(static_cast<size_t>(B) * static_cast<size_t>(Pd) * 4);
  w.total = off;
  return w;
}

// Square 2-D grid whose side splits into `levels` levels of 4 x 4 segments
// with a 32-point coarse map at every level.
int check_learn_grid(const uwb_grid* g, int levels) {
  if (levels < 1 || levels > 3) return fail(UWB_ERR_ARG, "levels %d not in [1, 3]", levels);
  if (g->dim != 2 || g->n[0] != g->n[1] || g->n[2] != 1)
    return fail(UWB_ERR_UNSUPPORTED, "the learned proposal needs a square 2-D grid");
  int need = cnn::MAP;
  for (int l = 1; l < levels; ++l) need *= cnn::SEG;
  if (g->n[0] % need != 0)
    return fail(UWB_ERR_UNSUPPORTED, "grid side %d is not a multiple of %d for %d level(s)",
                g->n[0], need, levels);
  return UWB_OK;
}

// One pass of the DAS image kernel over a 32 x 32 lattice per scan, written
// compactly to maps[B][32][32]: the uniform lattice `uni`, or per-scan boxes.
int run_map_pass(Device& dev, const Geo& geo, const float* traces, const float* ant,
                 long long ant_stride, const Variant& vm, int span, int use_tma,
                 const CUtensorMap* map, const LatBox* uni, const LatBox* boxes,
                 const int* prefix, float* maps, int* status, int step, cudaStream_t cs) {
  ImgParams p = base_params(geo, traces, ant, ant_stride, vm, span, use_tma, status);
  if (uni) {
    p.uni = *uni;
  } else {
    p.boxes = boxes;
    p.prefix = prefix;
    p.uni.tiles = 1;
  }
  p.compact = maps;
  p.compact_stride = cnn::MAP * cnn::MAP;
  const double dstep[3] = {static_cast<double>(step), static_cast<double>(step), 1.0};
  int cnt[3] = {cnn::MAP, cnn::MAP, 1};
  return run_image_kernel(dev, vm, p, map, static_cast<long long>(geo.B) * lattice_tiles(cnt, vm.tdim),
                          dstep, cs);
}

}  // namespace

extern "C" {

size_t uwb_coarse_maps_workspace(int batch) {
  if (batch < 1 || batch > (1 << 24)) return 0;
  return align256(static_cast<size_t>(batch) * sizeof(LatBox)) +
         align256(static_cast<size_t>(batch + 1) * 4);
}

int uwb_coarse_maps(int batch, const float* traces, int M, int N, const float* antennas,
                    long long antenna_stride, const uwb_grid* grid, double v, double fs,
                    int window, const int* region_lo, int side, float* maps, void* workspace,
                    size_t ws_bytes, void* stream) {
  Geo geo;
  int st = check_common(batch, traces, M, N, antennas, grid, v, fs, window, &geo);
  if (st) return st;
  if (!maps) return fail(UWB_ERR_ARG, "null maps");
  if (antenna_stride < 0) return fail(UWB_ERR_ARG, "negative antenna stride");
  if (grid->dim != 2 || grid->n[2] != 1) return fail(UWB_ERR_UNSUPPORTED, "coarse maps need a 2-D grid");
  if (side < cnn::MAP || side % cnn::MAP != 0 || side > grid->n[0] || side > grid->n[1])
    return fail(UWB_ERR_ARG, "side %d must be a multiple of %d within the grid", side, cnn::MAP);
  if (region_lo) {
    const size_t need = uwb_coarse_maps_workspace(batch);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || ws_bytes < need)
      return fail(UWB_ERR_WORKSPACE, "per-scan regions need %zu bytes of 256-byte aligned workspace",
                  need);
  }
  Device* dev;
  if ((st = device(&dev))) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  Variant vm;
  if ((st = pick_map_variant(M, window, &vm))) return st;
  const int span = pick_span(vm, M);
  CUtensorMap map;
  const int use_tma = encode_traces(geo, traces, span, &map);
  cudaError_t e = cudaMemsetAsync(maps, 0, static_cast<size_t>(batch) * cnn::MAP * cnn::MAP * 4, cs);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  const int step = side / cnn::MAP, o = (step - 1) / 2;
  if (!region_lo) {
    LatBox uni;
    const int lo[3] = {o, o, 0}, stp[3] = {step, step, 1}, cnt[3] = {cnn::MAP, cnn::MAP, 1};
    for (int a = 0; a < 3; ++a) {
      uni.lo[a] = lo[a];
      uni.step[a] = stp[a];
      uni.cnt[a] = cnt[a];
    }
    uni.tiles = lattice_tiles(uni.cnt, vm.tdim);
    return run_map_pass(*dev, geo, traces, antennas, antenna_stride, vm, span, use_tma, &map, &uni,
                        nullptr, nullptr, maps, dev->status, step, cs);
  }
  auto* boxes = static_cast<LatBox*>(workspace);
  auto* prefix = reinterpret_cast<int*>(static_cast<char*>(workspace) +
                                        align256(static_cast<size_t>(batch) * sizeof(LatBox)));
  if ((e = cnn::launch_region_boxes(region_lo, side, grid->n[0], batch, vm.tdim, boxes, dev->status,
                                    cs)) != cudaSuccess)
    return cuda_fail(e, "region boxes launch");
  if ((e = launch_plan(boxes, prefix, batch, cs)) != cudaSuccess) return cuda_fail(e, "plan launch");
  return run_map_pass(*dev, geo, traces, antennas, antenna_stride, vm, span, use_tma, &map, nullptr,
                      boxes, prefix, maps, dev->status, step, cs);
}

size_t uwb_localize_learned_workspace(int batch, const uwb_grid* grid, const uwb_rule* rule) {
  if (batch < 1 || batch > (1 << 24) || !grid || !rule || check_rule(rule)) return 0;
  if (grid->dim != 2) return 0;
  return learn_layout(batch, decimate(*grid, *rule).Pd).total;
}

int uwb_localize_learned(int batch, const float* traces, int M, int N, const float* antennas,
                         long long antenna_stride, const uwb_grid* grid, double v, double fs,
                         int window, int beamformer, const uwb_rule* rule, const void* packed,
                         float threshold, int levels, void* workspace, size_t ws_bytes,
                         uwb_result* out, void* stream) {
  Geo geo;
  int st = check_common(batch, traces, M, N, antennas, grid, v, fs, window, &geo);
  if (st) return st;
  if ((st = check_rule(rule))) return st;
  if ((st = check_learn_grid(grid, levels))) return st;
  if (!out || !packed) return fail(UWB_ERR_ARG, "null results or parameters");
  if (antenna_stride < 0) return fail(UWB_ERR_ARG, "negative antenna stride");
  if (!(threshold >= 0.f && threshold <= 1.f)) return fail(UWB_ERR_ARG, "threshold not in [0, 1]");
  const int bf = bf_of(beamformer);
  if (bf < 0) return fail(UWB_ERR_ARG, "unknown beamformer %d", beamformer);
  const Decim dc = decimate(geo.g, *rule);
  const LearnLayout L = learn_layout(batch, dc.Pd);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(UWB_ERR_WORKSPACE, "workspace must be non-null and 256-byte aligned");
  if (ws_bytes < L.total)
    return fail(UWB_ERR_WORKSPACE, "workspace of %zu bytes < %zu needed", ws_bytes, L.total);
  if ((st = umma_ready())) return st;
  Device* dev;
  if ((st = device(&dev))) return st;
  Variant vm, var;
  if ((st = pick_map_variant(M, window, &vm))) return st;
  if ((st = pick_variant(bf, M, window, 2, &var))) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  auto* keys = reinterpret_cast<unsigned long long*>(ws + L.keys);
  auto* status = reinterpret_cast<int*>(ws + L.status);
  auto* maps = reinterpret_cast<float*>(ws + L.maps);
  auto* scores = reinterpret_cast<float*>(ws + L.scores);
  auto* state = reinterpret_cast<LearnState*>(ws + L.state);
  auto* map_boxes = reinterpret_cast<LatBox*>(ws + L.map_boxes);
  auto* final_boxes = reinterpret_cast<LatBox*>(ws + L.final_boxes);
  auto* prof_boxes = reinterpret_cast<LatBox*>(ws + L.prof_boxes);
  auto* learned = reinterpret_cast<int*>(ws + L.learned);
  auto* prefix = reinterpret_cast<int*>(ws + L.prefix);
  auto* profile = reinterpret_cast<float*>(ws + L.profile);
  cudaError_t e = cudaMemsetAsync(ws + L.keys, 0, L.status + 4 - L.keys, cs);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(out, 0, static_cast<size_t>(batch) * sizeof(uwb_result), cs);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");

  const int span_m = pick_span(vm, M), span = pick_span(var, M);
  CUtensorMap map_m, map_f;
  const int tma_m = encode_traces(geo, traces, span_m, &map_m);
  const int tma_f = encode_traces(geo, traces, span, &map_f);
  const int ctas = cnn_ctas(*dev, batch);
  PhaseTimer timer(cs, kLearnedPhases);
  timer.mark();

  cnn::LearnParams lp;
  memset(&lp, 0, sizeof lp);
  lp.B = batch;
  lp.n = grid->n[0];
  lp.levels = levels;
  lp.threshold = threshold;
  lp.frame_num = rule->frame_num;
  lp.frame_den = rule->frame_den;
  lp.scores = scores;
  lp.state = state;
  lp.out = out;
  lp.map_boxes = map_boxes;
  lp.final_boxes = final_boxes;
  lp.prof_boxes = prof_boxes;
  lp.learned = learned;
  for (int a = 0; a < 3; ++a) {
    lp.doff[a] = dc.off[a];
    lp.dstep[a] = dc.step[a];
    lp.dcnt[a] = dc.cnt[a];
    lp.tdim_map[a] = vm.tdim[a];
    lp.tdim_final[a] = var.tdim[a];
  }

  // 1. the proposal, level by level: coarse DAS map, network, decision
  int side = grid->n[0];
  for (int level = 0; level < levels; ++level) {
    const int step = side / cnn::MAP;
    if (level == 0) {
      LatBox uni;
      const int o = (step - 1) / 2;
      for (int a = 0; a < 2; ++a) {
        uni.lo[a] = o;
        uni.step[a] = step;
        uni.cnt[a] = cnn::MAP;
      }
      uni.lo[2] = 0;
      uni.step[2] = 1;
      uni.cnt[2] = 1;
      uni.tiles = lattice_tiles(uni.cnt, vm.tdim);
      st = run_map_pass(*dev, geo, traces, antennas, antenna_stride, vm, span_m, tma_m, &map_m,
                        &uni, nullptr, nullptr, maps, status, step, cs);
    } else {
      if ((e = launch_plan(map_boxes, prefix, batch, cs)) != cudaSuccess)
        return cuda_fail(e, "plan launch");
      st = run_map_pass(*dev, geo, traces, antennas, antenna_stride, vm, span_m, tma_m, &map_m,
                        nullptr, map_boxes, prefix, maps, status, step, cs);
    }
    if (st) return st;
    if ((e = cnn::launch_forward(packed, maps, batch, scores, nullptr, nullptr, nullptr, status,
                                 ctas, cs)) != cudaSuccess)
      return cuda_fail(e, "network forward launch");
    if ((e = cnn::launch_decide(lp, level, cs)) != cudaSuccess) return cuda_fail(e, "decide launch");
    side /= cnn::SEG;
  }
  timer.mark();

  // 2. where the network was not confident: the decimated profile and the
  // Eq. 5 selection (Section III) for those scans only
  if ((e = launch_plan(prof_boxes, prefix, batch, cs)) != cudaSuccess)
    return cuda_fail(e, "plan launch");
  {
    ImgParams p1 = base_params(geo, traces, antennas, antenna_stride, var, span, tma_f, status);
    p1.boxes = prof_boxes;
    p1.prefix = prefix;
    p1.uni.tiles = 1;
    p1.compact = profile;
    p1.compact_stride = dc.Pd;
    const double dstep[3] = {static_cast<double>(dc.step[0]), static_cast<double>(dc.step[1]),
                             static_cast<double>(dc.step[2])};
    const int pc[3] = {dc.cnt[0], dc.cnt[1], dc.cnt[2]};
    if ((st = run_image_kernel(*dev, var, p1, &map_f,
                               static_cast<long long>(batch) * lattice_tiles(pc, var.tdim), dstep, cs)))
      return st;
  }
  SelParams sp;
  memset(&sp, 0, sizeof sp);
  sp.profile = profile;
  sp.prof_stride = dc.Pd;
  sp.B = batch;
  sp.dim = 2;
  for (int a = 0; a < 3; ++a) {
    sp.gn[a] = geo.g.n[a];
    sp.off[a] = dc.off[a];
    sp.step[a] = dc.step[a];
    sp.cnt[a] = dc.cnt[a];
    sp.tdim[a] = var.tdim[a];
  }
  sp.D = dc.D;
  sp.rule = *rule;
  sp.max_iters = dc.max_iters;
  sp.skip = learned;
  sp.boxes = final_boxes;
  sp.out = out;
  if ((e = launch_select(sp, cs)) != cudaSuccess) return cuda_fail(e, "select launch");
  if ((e = launch_plan(final_boxes, prefix, batch, cs)) != cudaSuccess)
    return cuda_fail(e, "plan launch");
  timer.mark();

  // 3. final region of every scan at full resolution + argmax
  {
    ImgParams p2 = base_params(geo, traces, antennas, antenna_stride, var, span, tma_f, status);
    p2.boxes = final_boxes;
    p2.prefix = prefix;
    p2.uni.tiles = 1;
    p2.keys = keys;
    int full_cnt[3] = {geo.g.n[0], geo.g.n[1], geo.g.n[2]};
    const double step1[3] = {1, 1, 1};
    if ((st = run_image_kernel(*dev, var, p2, &map_f,
                               static_cast<long long>(batch) * lattice_tiles(full_cnt, var.tdim), step1,
                               cs)))
      return st;
  }
  timer.mark();
  FinishParams fp;
  memset(&fp, 0, sizeof fp);
  fp.learn = state;
  fp.keys = keys;
  fp.boxes = final_boxes;
  fp.out = out;
  fp.B = batch;
  for (int a = 0; a < 3; ++a) {
    fp.gn[a] = geo.g.n[a];
    fp.org[a] = geo.g.origin[a];
    fp.pit[a] = geo.g.pitch[a];
  }
  fp.Pd = dc.Pd;
  if ((e = launch_finish(fp, status, cs)) != cudaSuccess) return cuda_fail(e, "finish launch");
  timer.mark();
  timer.commit();
  return UWB_OK;
}

}  // extern "C"

// ---- progressive re-evaluation (a variant of the ROI selection loop)
namespace {

struct ProgLayout {
  size_t keys, status, profile, lattice, state, next_boxes, final_boxes, prefix, total;
};

ProgLayout prog_layout(int B, long long Pd) {
  ProgLayout w;
  size_t off = 0;
  w.keys = off;
  off += static_cast<size_t>(B) * 8;
  w.status = off;
  off = align256(off + 4);
  w.profile = off;
  off += align256(static_cast<size_t>(B) * static_cast<size_t>(Pd) * 4);
  w.lattice = off;
  off += align256(static_cast<size_t>(B) * static_cast<size_t>(Pd) * 4);
  w.state = off;
  off += align256(static_cast<size_t>(B) * sizeof(ProgState));
  w.next_boxes = off;
  off += align256(static_cast<size_t>(B) * sizeof(LatBox));
  w.final_boxes = off;
  off += align256(static_cast<size_t>(B) * sizeof(LatBox));
  w.prefix = off;
  off += align256(static_cast<size_t>(B + 1) * 4);
  w.total = off;
  return w;
}

}  // namespace

extern "C" {

size_t uwb_localize_progressive_workspace(int batch, int M, int N, const uwb_grid* grid,
                                          int beamformer, const uwb_rule* rule) {
  if (batch < 1 || M < 1 || N < 1 || !grid || !rule || bf_of(beamformer) < 0 ||
      check_rule(rule))
    return 0;
  return prog_layout(batch, decimate(*grid, *rule).Pd).total;
}

int uwb_localize_progressive(int batch, const float* traces, int M, int N,
                             const float* antennas, long long antenna_stride,
                             const uwb_grid* grid, double v, double fs, int window,
                             int beamformer, const uwb_rule* rule, void* workspace,
                             size_t ws_bytes, uwb_result* out, void* stream) {
  Geo geo;
  int st = check_common(batch, traces, M, N, antennas, grid, v, fs, window, &geo);
  if (st) return st;
  if ((st = check_rule(rule))) return st;
  if (!out) return fail(UWB_ERR_ARG, "null result array");
  if (antenna_stride < 0) return fail(UWB_ERR_ARG, "negative antenna stride");
  const int bf = bf_of(beamformer);
  if (bf < 0) return fail(UWB_ERR_ARG, "unknown beamformer %d", beamformer);
  Variant var;
  if ((st = pick_variant(bf, M, window, geo.g.dim, &var))) return st;
  const Decim dc = decimate(geo.g, *rule);
  const ProgLayout L = prog_layout(batch, dc.Pd);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(UWB_ERR_WORKSPACE, "workspace must be non-null and 256-byte aligned");
  if (ws_bytes < L.total)
    return fail(UWB_ERR_WORKSPACE, "workspace of %zu bytes < %zu needed", ws_bytes, L.total);
  Device* dev;
  if ((st = device(&dev))) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  auto* keys = reinterpret_cast<unsigned long long*>(ws + L.keys);
  auto* status = reinterpret_cast<int*>(ws + L.status);
  auto* profile = reinterpret_cast<float*>(ws + L.profile);
  auto* lattice = reinterpret_cast<float*>(ws + L.lattice);
  auto* state = reinterpret_cast<ProgState*>(ws + L.state);
  auto* next_boxes = reinterpret_cast<LatBox*>(ws + L.next_boxes);
  auto* final_boxes = reinterpret_cast<LatBox*>(ws + L.final_boxes);
  auto* prefix = reinterpret_cast<int*>(ws + L.prefix);
  cudaError_t e = cudaMemsetAsync(ws + L.keys, 0, L.status + 4 - L.keys, cs);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  const int span = pick_span(var, M);
  CUtensorMap map;
  const int use_tma = encode_traces(geo, traces, span, &map);
  PhaseTimer timer(cs);
  timer.mark();

  // 1. the decimated profile (Section III, "Spatial Decimation")
  const double dstep[3] = {static_cast<double>(dc.step[0]), static_cast<double>(dc.step[1]),
                           static_cast<double>(dc.step[2])};
  const int pc[3] = {dc.cnt[0], dc.cnt[1], dc.cnt[2]};
  const long long lattice_work = static_cast<long long>(batch) * lattice_tiles(pc, var.tdim);
  {
    ImgParams p1 = base_params(geo, traces, antennas, antenna_stride, var, span, use_tma, status);
    for (int a = 0; a < 3; ++a) {
      p1.uni.lo[a] = dc.off[a];
      p1.uni.step[a] = dc.step[a];
      p1.uni.cnt[a] = dc.cnt[a];
    }
    p1.uni.tiles = lattice_tiles(p1.uni.cnt, var.tdim);
    p1.compact = profile;
    p1.compact_stride = dc.Pd;
    if ((st = run_image_kernel(*dev, var, p1, &map, lattice_work, dstep, cs))) return st;
  }
  timer.mark();

  // 2. the selection loop: one step kernel per iteration, each followed by
  // the image pass over every active scan's next region lattice
  ProgParams pp;
  memset(&pp, 0, sizeof pp);
  pp.profile = profile;
  pp.lattice = lattice;
  pp.stride = dc.Pd;
  pp.B = batch;
  pp.dim = geo.g.dim;
  for (int a = 0; a < 3; ++a) {
    pp.gn[a] = geo.g.n[a];
    pp.off[a] = dc.off[a];
    pp.step[a] = dc.step[a];
    pp.cnt[a] = dc.cnt[a];
    pp.tdim[a] = var.tdim[a];
  }
  pp.D = dc.D;
  pp.max_iters = dc.max_iters;
  pp.rule = *rule;
  pp.state = state;
  pp.next_boxes = next_boxes;
  pp.final_boxes = final_boxes;
  pp.out = out;
  for (int it = 1; it <= dc.max_iters; ++it) {
    if ((e = launch_prog_step(pp, it, cs)) != cudaSuccess) return cuda_fail(e, "step launch");
    if (it == dc.max_iters) break;
    if ((e = launch_plan(next_boxes, prefix, batch, cs)) != cudaSuccess)
      return cuda_fail(e, "plan launch");
    ImgParams pl = base_params(geo, traces, antennas, antenna_stride, var, span, use_tma, status);
    pl.boxes = next_boxes;
    pl.prefix = prefix;
    pl.uni.tiles = 1;
    pl.compact = lattice;
    pl.compact_stride = dc.Pd;
    if ((st = run_image_kernel(*dev, var, pl, &map, lattice_work, dstep, cs))) return st;
  }
  if ((e = launch_plan(final_boxes, prefix, batch, cs)) != cudaSuccess)
    return cuda_fail(e, "plan launch");
  timer.mark();

  // 3. final region at full resolution + argmax
  {
    ImgParams p2 = base_params(geo, traces, antennas, antenna_stride, var, span, use_tma, status);
    p2.boxes = final_boxes;
    p2.prefix = prefix;
    p2.uni.tiles = 1;
    p2.keys = keys;
    int full_cnt[3] = {geo.g.n[0], geo.g.n[1], geo.g.n[2]};
    const double step1[3] = {1, 1, 1};
    if ((st = run_image_kernel(*dev, var, p2, &map,
                               static_cast<long long>(batch) * lattice_tiles(full_cnt, var.tdim), step1,
                               cs)))
      return st;
  }
  timer.mark();
  FinishParams fp;
  memset(&fp, 0, sizeof fp);
  fp.prog = state;
  fp.keys = keys;
  fp.boxes = final_boxes;
  fp.out = out;
  fp.B = batch;
  for (int a = 0; a < 3; ++a) {
    fp.gn[a] = geo.g.n[a];
    fp.org[a] = geo.g.origin[a];
    fp.pit[a] = geo.g.pitch[a];
  }
  fp.Pd = dc.Pd;
  if ((e = launch_finish(fp, status, cs)) != cudaSuccess) return cuda_fail(e, "finish launch");
  timer.mark();
  timer.commit();
  return UWB_OK;
}

}  // extern "C"

extern "C" {

int uwb_measure_peaks(double* fp32_tflops, double* shared_wavefronts_per_s) {
  if (!fp32_tflops || !shared_wavefronts_per_s) return fail(UWB_ERR_ARG, "null output");
  Device* dev;
  int st = device(&dev);
  if (st) return st;
  cudaError_t e = measure_peaks(dev->sms, fp32_tflops, shared_wavefronts_per_s);
  return e == cudaSuccess ? UWB_OK : cuda_fail(e, "peak microbenchmarks");
}

int uwb_wait_selftest(int probes) {
  if (probes < 1 || probes > (1 << 24))
    return fail(UWB_ERR_ARG, "probes must lie in 1 .. 2^24 (got %d)", probes);
  Device* dev;
  int st = device(&dev);
  if (st) return st;
  const cudaError_t e = wait_selftest(dev->status, probes);
  return e == cudaSuccess ? UWB_OK : cuda_fail(e, "bounded-wait self-check");
}

}  // extern "C"
