// Learned segment proposal on the 5th-generation tensor cores: the network's
// forward, backward and Adam kernels, a tensor-core self-check, and the
// per-scan decisions of the learned localisation.
//
// Not part of the paper: the network proposes the segments that Section III's
// ROI selection would otherwise choose with the Eq. 5 metric, and that metric
// decides instead whenever the network is not confident.
//
// Convolutions as implicit GEMMs without an im2col copy. An activation map of
// 32 channels lives in shared memory as 4 groups of 8 channels; inside a group
// every position is one 16-byte row, positions run along padded map rows of 33
// (one zero column), with 34 zero positions before the map and zeros after
// it. In that layout a block of 128 consecutive positions, shifted by a tap's
// offset dy * 33 + dx, is a K-major tcgen05 operand (rows = positions, K = the
// 8-channel groups) that only needs a different start address; the zero
// column and the zero margins supply the convolution's zero padding. One
// layer is then 9 tiles x 9 taps x 2 K-steps of M = 128, N = 32, K = 16 BF16
// MMAs accumulating in TMEM (FP32), and the epilogue adds the bias, applies
// the ReLU and writes the next layer's BF16 map in the same layout.
#include <cuda_bf16.h>

#include "ptx.cuh"
#include "umma.cuh"
#include "uwb_internal.cuh"

namespace uwb {
namespace cnn {
namespace {

constexpr long kProbes = 1L << 24;  // bounded MMA-completion waits
constexpr uint32_t kIdesc = umma_idesc_bf16(128, CH);
constexpr int THREADS = 256;
constexpr int TMEM_COLS = 512;      // TILES x 32 FP32 columns, rounded to a power of two
constexpr int WTAP = 2048;          // one tap's 32 x 32 BF16 weight operand
constexpr int WOP_BYTES = TAPS * WTAP;

static_assert(TILES * CH <= TMEM_COLS, "accumulators exceed the TMEM allocation");
static_assert((TILES - 1) * 128 + 127 + 2 * PAD0 < U, "operand rows leave the buffer");

// byte offset of channel c of buffer position u
__host__ __device__ constexpr int act_off(int u, int c) {
  return (c >> 3) * LBO_ACT + u * 16 + (c & 7) * 2;
}
__host__ __device__ constexpr int pos_u(int y, int x) { return PAD0 + y * Q + x; }
// position offset of tap t = 3 (dy + 1) + (dx + 1)
__host__ __device__ constexpr int tap_shift(int t) { return (t / 3 - 1) * Q + (t % 3 - 1); }
// K-major operand of one tap: row n (output channel of the GEMM), column k
__host__ __device__ constexpr int wop_off(int t, int n, int k) {
  return t * WTAP + (k >> 3) * 512 + (n >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ float bf2f(uint32_t h) { return __uint_as_float(h << 16); }

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void copy16(void* dst, const void* src, int bytes) {
  uint4* d = static_cast<uint4*>(dst);
  const uint4* s = static_cast<const uint4*>(src);
  for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = s[i];
}

// Thread 0 waits for the MMA-completion phase; every thread learns whether it
// came. After a timeout the status word is set and the MMAs get a second
// bounded wait before the caller frees the TMEM they write.
__device__ __forceinline__ bool wait_mma(uint64_t* bar, uint32_t phase, int* status) {
  int late = 0;
  if (threadIdx.x == 0) {
    uint32_t ok = 0;
    for (long it = 0; it < kProbes && !ok; ++it) ok = mbar_try_wait(bar, phase);
    if (!ok) {
      late = 1;
      if (status) atomicExch(status, UWB_ERR_TIMEOUT);
      for (long it = 0; it < kProbes && !ok; ++it) ok = mbar_try_wait(bar, phase);
    }
  }
  return !__syncthreads_or(late);
}

// One 3x3 convolution layer (32 -> 32 channels) into TMEM: tile i's
// accumulator is columns [32 i, 32 i + 32). The descriptors are built once;
// each MMA adds its operand's byte offset / 16 to the 14-bit address field,
// which stays inside [0, 2^14) for every operand of the layer (shared-memory
// addresses are below 256 KB and all offsets land inside the buffers), so
// nothing carries into the stride fields. This thread issues tiles first,
// first + stride, ...: each tile's 18 MMAs, then an arrive on bars[i] once
// they (and every earlier MMA of this thread) have completed, so that tile
// i's epilogue can run while the tensor cores compute later tiles.
__device__ __forceinline__ void issue_conv_tiles(uint32_t in_base, uint32_t w_base, uint32_t tmem,
                                                 uint64_t* bars, int first, int stride) {
  const uint64_t a0 = umma_desc(in_base + PAD0 * 16, LBO_ACT, 128);
  const uint64_t b0 = umma_desc(w_base, 512, 128);
#pragma unroll 1
  for (int i = first; i < TILES; i += stride) {
    const uint64_t ai = a0 + static_cast<uint64_t>(i * 128);
    const uint32_t d = tmem + i * CH;
#pragma unroll
    for (int t = 0; t < TAPS; ++t)
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const int64_t da = (ks * 2 * LBO_ACT) / 16 + tap_shift(t);
        const uint64_t b = b0 + static_cast<uint64_t>((t * WTAP + ks * 2 * 512) / 16);
        umma_bf16(d, ai + static_cast<uint64_t>(da), b, kIdesc, (t | ks) != 0);
      }
    umma_commit(bars + i);
  }
}

// One warp's bounded wait for a phase of `bar`: lane 0 polls, the warp learns
// whether it came.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t phase, int lane) {
  uint32_t ok = 0;
  if (lane == 0)
    for (long it = 0; it < kProbes && !ok; ++it) ok = mbar_try_wait(bar, phase);
  return __shfl_sync(0xFFFFFFFFu, ok, 0) != 0;
}

// ---------------------------------------------------------------- self-check
// D[128][32] = A[128][64] B[32][64]^T through the same descriptor and TMEM
// conventions as the network. Operand areas are sized so that every address
// the MMA can form stays inside them even if the two descriptor strides were
// read the other way round (then the result is wrong, and the check says so).
constexpr int ST_A = 0, ST_B = 49152, ST_BAR = 57344, ST_SLOT = 57352, ST_SMEM = 57360;

__global__ void __launch_bounds__(128) k_umma_selftest(const uint16_t* A, const uint16_t* Bm,
                                                       float* D, int* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + ST_BAR);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + ST_SLOT);
  for (int i = tid; i < ST_BAR / 16; i += 128) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  for (int i = tid; i < 128 * 64; i += 128) {
    const int m = i >> 6, k = i & 63;
    *reinterpret_cast<uint16_t*>(sm + ST_A + (k >> 3) * 2048 + (m >> 3) * 128 + (m & 7) * 16 +
                                 (k & 7) * 2) = A[i];
  }
  for (int i = tid; i < 32 * 64; i += 128) {
    const int n = i >> 6, k = i & 63;
    *reinterpret_cast<uint16_t*>(sm + ST_B + (k >> 3) * 512 + (n >> 3) * 128 + (n & 7) * 16 +
                                 (k & 7) * 2) = Bm[i];
  }
  if (tid == 0) mbar_init(bar, 1);
  if (warp == 0) tmem_alloc(slot, 256);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  if (tid == 0) {
    for (int ks = 0; ks < 4; ++ks)
      umma_bf16(tmem, umma_desc(smem_u32(sm + ST_A) + ks * 2 * 2048, 2048, 128),
                umma_desc(smem_u32(sm + ST_B) + ks * 2 * 512, 512, 128), kIdesc, ks > 0);
    umma_commit(bar);
  }
  if (wait_mma(bar, 0, status)) {
    tc_fence_after();
    float v[32];
    tmem_ld32(tmem + (static_cast<uint32_t>(warp * 32) << 16), v);
#pragma unroll
    for (int j = 0; j < 32; ++j) D[(warp * 32 + lane) * 32 + j] = v[j];
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 256);
  }
}

// ---------------------------------------------------------------- forward
// Shared memory of the forward kernel (bytes).
constexpr int F_ACT0 = 0;
constexpr int F_ACT1 = F_ACT0 + ACT_BYTES;
constexpr int F_W2 = F_ACT1 + ACT_BYTES;
constexpr int F_W3 = F_W2 + WOP_BYTES;
constexpr int F_X = F_W3 + WOP_BYTES;          // X0, float, buffer positions
constexpr int W1_ROW = 12;                     // W1 rows padded to 3 float4
constexpr int F_W1 = F_X + U * 4;              // W1 as float [32][12]
constexpr int F_BIAS = F_W1 + CH * W1_ROW * 4; // b1, b2, b3, wh [32] each, bh
constexpr int F_F = F_BIAS + 144 * 4;          // segment means, [32 channels][16 segments]
constexpr int F_RED = F_F + SEGS * CH * 4;     // reduction scratch [16]
constexpr int F_BAR = F_RED + 64;              // one mbarrier per tile
constexpr int F_SLOT = F_BAR + 8 * 16;
constexpr int F_SMEM = F_SLOT + 8;
static_assert(F_W2 % 16 == 0 && F_W3 % 16 == 0 && F_X % 16 == 0 && F_BAR % 8 == 0, "alignment");

// The forward kernel runs 16 warps. One lane of each of warps 0-3 (one warp
// per scheduler) issues the MMAs of tiles w, w + 4, ...: with N = 32 output
// channels each MMA is short, and one issuing thread left the tensor pipe
// idle between them (162 MMAs per layer took 4.0 us from one thread, 5.9 us
// beside polling epilogue warps, 4.0 us from four threads while the
// epilogues of finished tiles run). Warps 4-15 are three epilogue groups of
// four, group g taking tiles g, g + 3, g + 6 of a layer, each as soon as its
// own commit has arrived; every warp takes part in the CUDA-core work
// (normalisation, layer 1, segment means).
constexpr int F_THREADS = 512;
constexpr int F_WARPS = F_THREADS / 32;
static_assert(F_WARPS * 2 <= 64 && TILES == 9, "reduction scratch and epilogue groups");

// Epilogue of a forward layer for this warp's tiles: TMEM tile rows + bias,
// ReLU, BF16 -> `out`. A warp reads the TMEM lane quarter (warp % 4), i.e.
// tile rows 32 (warp % 4) + lane. Returns false if a tile's commit did not
// arrive within the bounded wait.
__device__ __forceinline__ bool epilogue_relu(unsigned char* out, const float* bias,
                                              uint32_t tmem, uint64_t* bars, uint32_t phase,
                                              int warp, int lane) {
  if (warp < 4) return true;
  const int q = warp & 3;
  for (int i = (warp >> 2) - 1; i < TILES; i += 3) {
    if (!warp_wait(bars + i, phase, lane)) return false;
    tc_fence_after();
    float v[32];
    tmem_ld32(tmem + (static_cast<uint32_t>(q * 32) << 16) + i * CH, v);
    const int p = i * 128 + q * 32 + lane;
    if (p < NPOS && p % Q < MAP) {
      uint32_t w[16];
#pragma unroll
      for (int c = 0; c < 32; c += 2)
        w[c >> 1] = pack2(fmaxf(v[c] + bias[c], 0.f), fmaxf(v[c + 1] + bias[c + 1], 0.f));
#pragma unroll
      for (int g = 0; g < 4; ++g)
        *reinterpret_cast<uint4*>(out + act_off(PAD0 + p, 8 * g)) =
            make_uint4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3]);
    }
  }
  return true;
}

__global__ void __launch_bounds__(F_THREADS, 1)
    k_cnn_forward(const unsigned char* __restrict__ packed, const float* __restrict__ maps,
                  int B, float* __restrict__ scores, const int* __restrict__ labels,
                  unsigned char* __restrict__ save, float* __restrict__ loss, int* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* act0 = sm + F_ACT0;
  unsigned char* act1 = sm + F_ACT1;
  float* sX = reinterpret_cast<float*>(sm + F_X);
  float* sW1 = reinterpret_cast<float*>(sm + F_W1);
  float* sBias = reinterpret_cast<float*>(sm + F_BIAS);
  float* sF = reinterpret_cast<float*>(sm + F_F);
  float* sRed = reinterpret_cast<float*>(sm + F_RED);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + F_BAR);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + F_SLOT);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // the padding of both maps and of X0 stays zero for the whole kernel
  for (int i = tid; i < 2 * ACT_BYTES / 16; i += F_THREADS)
    reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < U; i += F_THREADS) sX[i] = 0.f;
  const uint16_t* pw1 = reinterpret_cast<const uint16_t*>(packed + PK_W1);
  const uint16_t* pw2 = reinterpret_cast<const uint16_t*>(packed + PK_W2);
  const uint16_t* pw3 = reinterpret_cast<const uint16_t*>(packed + PK_W3);
  const float* pf = reinterpret_cast<const float*>(packed + PK_F32);
  for (int i = tid; i < CH * W1_ROW; i += F_THREADS) {
    const int c = i / W1_ROW, t = i % W1_ROW;
    sW1[i] = t < TAPS ? bf2f(pw1[c * TAPS + t]) : 0.f;
  }
  for (int i = tid; i < 4 * CH + 1; i += F_THREADS) sBias[i] = pf[i];
  for (int i = tid; i < CH * TAPS * CH; i += F_THREADS) {
    const int o = i / (TAPS * CH), t = (i / CH) % TAPS, c = i % CH;  // W[o][t][c]
    *reinterpret_cast<uint16_t*>(sm + F_W2 + wop_off(t, o, c)) = pw2[i];
    *reinterpret_cast<uint16_t*>(sm + F_W3 + wop_off(t, o, c)) = pw3[i];
  }
  if (tid < TILES) mbar_init(bar + tid, 1);
  if (warp == 0) tmem_alloc(slot, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  uint32_t phase = 0;

  // each map's energies are loaded one map ahead
  constexpr int PER = MAP * MAP / F_THREADS;  // map points per thread
  float e_next[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j) e_next[j] = 0.f;
  if (blockIdx.x < B)
#pragma unroll
    for (int j = 0; j < PER; ++j)
      e_next[j] = maps[static_cast<size_t>(blockIdx.x) * (MAP * MAP) + tid + F_THREADS * j];

  for (int b = blockIdx.x; b < B; b += gridDim.x) {
    unsigned char* sv = save ? save + static_cast<size_t>(b) * SAVE_BYTES : nullptr;
    // ---- X0 = E / max E (all-zero maps stay zero; non-finite values are
    // recorded and read as zero)
    float e[PER], mx = 0.f;
#pragma unroll
    for (int j = 0; j < PER; ++j) e[j] = e_next[j];
    if (b + static_cast<int>(gridDim.x) < B)
#pragma unroll
      for (int j = 0; j < PER; ++j)
        e_next[j] = maps[static_cast<size_t>(b + gridDim.x) * (MAP * MAP) + tid + F_THREADS * j];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      if (!isfinite(e[j])) {
        if (status) atomicExch(status, UWB_ERR_NONFINITE);
        e[j] = 0.f;
      }
      mx = fmaxf(mx, e[j]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    if (lane == 0) sRed[warp] = mx;
    __syncthreads();
    mx = sRed[0];
    for (int w = 1; w < F_WARPS; ++w) mx = fmaxf(mx, sRed[w]);
    const float scale = mx > 0.f ? 1.0f / mx : 0.f;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int p = tid + F_THREADS * j;
      sX[pos_u(p >> 5, p & 31)] = e[j] * scale;
    }
    __syncthreads();
    if (sv) copy16(sv + SAVE_X0, sX, U * 4);

    // ---- layer 1 (1 -> 32 channels) on the CUDA cores: this thread's two
    // positions as the lanes of paired multiply-adds (each lane the same
    // fused multiply-adds in the same order as one position alone), so that
    // every weight is read once per two positions
    static_assert(PER == 2, "layer 1 pairs the thread's two positions");
    {
      float2 xv[TAPS];
      int uu[PER];
#pragma unroll
      for (int j = 0; j < PER; ++j) {
        const int p = tid + F_THREADS * j;
        uu[j] = pos_u(p >> 5, p & 31);
      }
#pragma unroll
      for (int t = 0; t < TAPS; ++t)
        xv[t] = make_float2(sX[uu[0] + tap_shift(t)], sX[uu[1] + tap_shift(t)]);
#pragma unroll 1
      for (int g = 0; g < 4; ++g) {
        uint32_t w[PER][4];
#pragma unroll
        for (int c2 = 0; c2 < 4; ++c2) {
          float2 z[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int c = 8 * g + 2 * c2 + h;
            const float4* wr = reinterpret_cast<const float4*>(sW1 + c * W1_ROW);
            const float4 q0 = wr[0], q1 = wr[1], q2 = wr[2];
            const float wt[TAPS] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x};
            float2 acc = make_float2(sBias[c], sBias[c]);
#pragma unroll
            for (int t = 0; t < TAPS; ++t) acc = __ffma2_rn(make_float2(wt[t], wt[t]), xv[t], acc);
            z[h] = make_float2(fmaxf(acc.x, 0.f), fmaxf(acc.y, 0.f));
          }
          w[0][c2] = pack2(z[0].x, z[1].x);
          w[1][c2] = pack2(z[0].y, z[1].y);
        }
#pragma unroll
        for (int j = 0; j < PER; ++j)
          *reinterpret_cast<uint4*>(act0 + act_off(uu[j], 8 * g)) =
              make_uint4(w[j][0], w[j][1], w[j][2], w[j][3]);
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (sv) copy16(sv + SAVE_A1, act0, ACT_BYTES);

    // ---- layers 2 and 3 on the tensor cores: act0 -> act1 -> act0
    bool alive = true;
    for (int l = 0; l < 2 && alive; ++l) {
      unsigned char* in = l == 0 ? act0 : act1;
      unsigned char* out = l == 0 ? act1 : act0;
      if (warp < 4 && lane == 0) {
        tc_fence_after();
        issue_conv_tiles(smem_u32(in), smem_u32(sm + (l == 0 ? F_W2 : F_W3)), tmem, bar, warp, 4);
      }
      const bool ok = epilogue_relu(out, sBias + CH * (l + 1), tmem, bar, phase, warp, lane);
      tc_fence_before();
      fence_proxy_async_smem();
      alive = !__syncthreads_or(!ok);
      if (!alive) {
        // a commit did not arrive in time: record it, give the MMAs a last
        // bounded chance to complete (they write the TMEM freed below), stop
        if (tid == 0) {
          if (status) atomicExch(status, UWB_ERR_TIMEOUT);
          for (int i = 0; i < TILES; ++i) {  // every issuing thread's last commit among them
            uint32_t done = 0;
            for (long it = 0; it < kProbes && !done; ++it) done = mbar_try_wait(bar + i, phase);
          }
        }
        __syncthreads();
        break;
      }
      phase ^= 1u;
      if (sv) copy16(sv + (l == 0 ? SAVE_A2 : SAVE_A3), out, ACT_BYTES);
    }
    if (!alive) break;

    // ---- segment means F[s][c] of A3 (in act0): thread = (segment s,
    // 8-channel group g, segment row r); the 8 rows of a (s, g) are
    // neighbouring lanes and are summed with shuffles
    {
      const int r = tid & 7, g = (tid >> 3) & 3, s = tid >> 5, sy = s >> 2, sx = s & 3;
      float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      {
        const int iy = r;
#pragma unroll
        for (int ix = 0; ix < 8; ++ix) {
          const uint4 v = *reinterpret_cast<const uint4*>(
              act0 + act_off(pos_u(8 * sy + iy, 8 * sx + ix), 8 * g));
          const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            acc[2 * k] += bf2f(wv[k] & 0xFFFFu);
            acc[2 * k + 1] += bf2f(wv[k] >> 16);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        acc[k] += __shfl_xor_sync(0xFFFFFFFFu, acc[k], 1);
        acc[k] += __shfl_xor_sync(0xFFFFFFFFu, acc[k], 2);
        acc[k] += __shfl_xor_sync(0xFFFFFFFFu, acc[k], 4);
      }
      if (r == 0)
#pragma unroll
        for (int k = 0; k < 8; ++k) sF[(8 * g + k) * SEGS + s] = acc[k] * (1.0f / 64.0f);
    }
    __syncthreads();

    // ---- head, softmax, loss
    if (warp == 0) {
      float z = -INFINITY;
      if (lane < SEGS) {
        z = sBias[4 * CH];
        for (int c = 0; c < CH; ++c) z = fmaf(sBias[3 * CH + c], sF[c * SEGS + lane], z);
        if (scores) scores[static_cast<size_t>(b) * SEGS + lane] = z;
      }
      if (labels) {
        float m = z;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
        const float ex = lane < SEGS ? expf(z - m) : 0.f;
        float sum = ex;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
        const int lab = labels[b];
        if (lane < SEGS) {
          const float p = ex / sum;
          float* dz = reinterpret_cast<float*>(sv + SAVE_DZ);
          dz[lane] = (p - (lane == lab ? 1.f : 0.f)) / static_cast<float>(B);
          if (lane == lab) atomicAdd(loss, (logf(sum) - (z - m)) / static_cast<float>(B));
        }
      }
    }
    if (sv)
      for (int i = tid; i < SEGS * CH; i += F_THREADS)
        reinterpret_cast<float*>(sv + SAVE_F)[i] = sF[(i % CH) * SEGS + i / CH];  // F[s][c]
    __syncthreads();
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ---------------------------------------------------------------- backward
// The backward pass runs on the CUDA cores (BF16 operands, FP32 sums): per
// map, the weight gradient of each 32 -> 32 layer and the input gradient
// G_{l-1} = bf16(conv^T(G_l; W_l) ⊙ [A_{l-1} > 0]). A tensor-core version of
// the input gradient (the forward loop with negated offsets) raised an
// illegal-instruction fault on the GB300 whose cause was not found.
constexpr int G_G = 0;                          // gradient map G_l (BF16, padded layout)
constexpr int G_X = G_G + ACT_BYTES;            // the layer's input A_{l-1}
constexpr int G_W3 = G_X + ACT_BYTES;           // W3, W2 as BF16 [tap][c_out][c_in]
constexpr int G_W2 = G_W3 + CH * TAPS * CH * 2;
constexpr int G_X0 = G_W2 + CH * TAPS * CH * 2; // X0, float
constexpr int G_DZ = G_X0 + U * 4;              // dz [16]
constexpr int G_WH = G_DZ + 64;                 // wh [32]
constexpr int G_SMEM = G_WH + 128;
static_assert(G_W3 % 16 == 0 && G_X0 % 16 == 0, "alignment");

// Input gradient of one layer for this warp's 128 map positions, input
// channel c = lane: sum over taps and output channels of G_l at the position
// shifted back by the tap times W[o][t][c], masked by the layer input `x`,
// rounded to BF16 and written into `out` (a padded map in global memory).
__device__ __forceinline__ void input_grad(const unsigned char* g, const uint16_t* w,
                                           const unsigned char* x, unsigned char* out, int warp,
                                           int lane) {
  for (int pb = warp * 128; pb < warp * 128 + 128; pb += 8) {
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int t = 0; t < TAPS; ++t) {
      float wv[CH];
#pragma unroll
      for (int o = 0; o < CH; ++o) wv[o] = bf2f(w[(t * CH + o) * CH + lane]);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int pv = pb + j;
        const int u = pos_u(pv >> 5, pv & 31) - tap_shift(t);
#pragma unroll
        for (int gr = 0; gr < 4; ++gr) {
          const uint4 q = *reinterpret_cast<const uint4*>(g + act_off(u, 8 * gr));
          const uint32_t qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            acc[j] = fmaf(bf2f(qv[k] & 0xFFFFu), wv[8 * gr + 2 * k], acc[j]);
            acc[j] = fmaf(bf2f(qv[k] >> 16), wv[8 * gr + 2 * k + 1], acc[j]);
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int pv = pb + j;
      const int u = pos_u(pv >> 5, pv & 31);
      const uint32_t a = *reinterpret_cast<const uint16_t*>(x + act_off(u, lane));
      const float gv = (a & 0x7FFFu) && !(a & 0x8000u) ? acc[j] : 0.f;
      *reinterpret_cast<__nv_bfloat16*>(out + act_off(u, lane)) = __float2bfloat16_rn(gv);
    }
  }
}

// dW[o][t][c] += sum_u G[u][o] X[u + shift(t)][c] for this thread's 4 output
// channels o = 4 (warp) + j and input channel c = lane; db[o] += sum_u G[u][o].
__device__ __forceinline__ void weight_grad(const unsigned char* g, const unsigned char* x,
                                            float (&acc)[TAPS * 4], float (&accb)[4], int warp,
                                            int lane) {
  const int o0 = 4 * warp;
#pragma unroll 2
  for (int p = 0; p < NPOS; ++p) {
    const int u = PAD0 + p;
    const uint2 gg = *reinterpret_cast<const uint2*>(g + act_off(u, o0));
    const float gv[4] = {bf2f(gg.x & 0xFFFFu), bf2f(gg.x >> 16), bf2f(gg.y & 0xFFFFu),
                         bf2f(gg.y >> 16)};
#pragma unroll
    for (int j = 0; j < 4; ++j) accb[j] += gv[j];
#pragma unroll
    for (int t = 0; t < TAPS; ++t) {
      const float a =
          bf2f(*reinterpret_cast<const uint16_t*>(x + act_off(u + tap_shift(t), lane)));
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[t * 4 + j] = fmaf(gv[j], a, acc[t * 4 + j]);
    }
  }
}

// Consumes the training record: its A3 and A2 slots are overwritten by G2 and
// G1 (same padded layout, zero padding kept).
__global__ void __launch_bounds__(THREADS, 1)
    k_cnn_backward(const unsigned char* __restrict__ packed, unsigned char* __restrict__ save,
                   int B, float* __restrict__ grad) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* sG = sm + G_G;
  unsigned char* sXa = sm + G_X;
  uint16_t* sW3 = reinterpret_cast<uint16_t*>(sm + G_W3);
  uint16_t* sW2 = reinterpret_cast<uint16_t*>(sm + G_W2);
  float* sX0 = reinterpret_cast<float*>(sm + G_X0);
  float* sDz = reinterpret_cast<float*>(sm + G_DZ);
  float* sWh = reinterpret_cast<float*>(sm + G_WH);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (int i = tid; i < ACT_BYTES / 16; i += THREADS)
    reinterpret_cast<uint4*>(sG)[i] = make_uint4(0, 0, 0, 0);
  const uint16_t* pw2 = reinterpret_cast<const uint16_t*>(packed + PK_W2);
  const uint16_t* pw3 = reinterpret_cast<const uint16_t*>(packed + PK_W3);
  const float* pf = reinterpret_cast<const float*>(packed + PK_F32);
  for (int i = tid; i < CH * TAPS * CH; i += THREADS) {
    const int o = i / (TAPS * CH), t = (i / CH) % TAPS, c = i % CH;  // W[o][t][c]
    sW3[(t * CH + o) * CH + c] = pw3[i];
    sW2[(t * CH + o) * CH + c] = pw2[i];
  }
  if (tid < CH) sWh[tid] = pf[3 * CH + tid];
  __syncthreads();

  float accW3[TAPS * 4] = {}, accW2[TAPS * 4] = {}, accW1[TAPS] = {};
  float accB3[4] = {}, accB2[4] = {}, accB1 = 0.f, accWh = 0.f, accBh = 0.f;

  for (int b = blockIdx.x; b < B; b += gridDim.x) {
    unsigned char* sv = save + static_cast<size_t>(b) * SAVE_BYTES;
    const float* Fg = reinterpret_cast<const float*>(sv + SAVE_F);
    if (tid < SEGS) sDz[tid] = reinterpret_cast<const float*>(sv + SAVE_DZ)[tid];
    __syncthreads();
    // ---- head: dwh[c] = sum_s dz[s] F[s][c], dbh = sum_s dz[s]
    if (tid < CH) {
      float a = 0.f;
      for (int s = 0; s < SEGS; ++s) a = fmaf(sDz[s], Fg[s * CH + tid], a);
      accWh += a;
    }
    if (tid == 0)
      for (int s = 0; s < SEGS; ++s) accBh += sDz[s];
    // ---- G3 = bf16(dz[seg] wh[c] / 64 ⊙ [A3 > 0])
    for (int p = tid; p < MAP * MAP; p += THREADS) {
      const int y = p >> 5, x = p & 31, u = pos_u(y, x);
      const float d = sDz[4 * (y >> 3) + (x >> 3)] * (1.0f / 64.0f);
#pragma unroll
      for (int gr = 0; gr < 4; ++gr) {
        const uint4 a = *reinterpret_cast<const uint4*>(sv + SAVE_A3 + act_off(u, 8 * gr));
        const uint32_t av[4] = {a.x, a.y, a.z, a.w};
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int c = 8 * gr + 2 * k;
          const float lo = (av[k] & 0x7FFFu) && !(av[k] & 0x8000u) ? d * sWh[c] : 0.f;
          const float hi =
              ((av[k] >> 16) & 0x7FFFu) && !(av[k] >> 31) ? d * sWh[c + 1] : 0.f;
          w[k] = pack2(lo, hi);
        }
        *reinterpret_cast<uint4*>(sG + act_off(u, 8 * gr)) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    copy16(sXa, sv + SAVE_A2, ACT_BYTES);
    __syncthreads();

    // ---- layer 3: dW3, db3; G2 -> the record's A3 slot
    weight_grad(sG, sXa, accW3, accB3, warp, lane);
    input_grad(sG, sW3, sXa, sv + SAVE_A3, warp, lane);
    __syncthreads();
    __threadfence_block();
    copy16(sG, sv + SAVE_A3, ACT_BYTES);
    copy16(sXa, sv + SAVE_A1, ACT_BYTES);
    __syncthreads();

    // ---- layer 2: dW2, db2; G1 -> the record's A2 slot
    weight_grad(sG, sXa, accW2, accB2, warp, lane);
    input_grad(sG, sW2, sXa, sv + SAVE_A2, warp, lane);
    __syncthreads();
    __threadfence_block();
    copy16(sG, sv + SAVE_A2, ACT_BYTES);
    copy16(sX0, sv + SAVE_X0, U * 4);
    __syncthreads();

    // ---- layer 1: dW1[o][t] = sum_u G1[u][o] X0[u + shift(t)], db1
    {
      const int o = lane;
      const int per = (NPOS + 7) / 8;
      const int p0 = warp * per, p1 = min(NPOS, p0 + per);
      for (int p = p0; p < p1; ++p) {
        const int u = PAD0 + p;
        const float gv = bf2f(*reinterpret_cast<const uint16_t*>(sG + act_off(u, o)));
        accB1 += gv;
#pragma unroll
        for (int t = 0; t < TAPS; ++t) accW1[t] = fmaf(gv, sX0[u + tap_shift(t)], accW1[t]);
      }
    }
    __syncthreads();
  }

  // ---- flush this CTA's sums (grad layout = parameter layout)
#pragma unroll
  for (int t = 0; t < TAPS; ++t)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int o = 4 * warp + j;
      atomicAdd(grad + TH_W3 + (o * TAPS + t) * CH + lane, accW3[t * 4 + j]);
      atomicAdd(grad + TH_W2 + (o * TAPS + t) * CH + lane, accW2[t * 4 + j]);
    }
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      atomicAdd(grad + TH_B3 + 4 * warp + j, accB3[j]);
      atomicAdd(grad + TH_B2 + 4 * warp + j, accB2[j]);
    }
#pragma unroll
  for (int t = 0; t < TAPS; ++t) atomicAdd(grad + TH_W1 + lane * TAPS + t, accW1[t]);
  atomicAdd(grad + TH_B1 + lane, accB1);
  if (tid < CH) atomicAdd(grad + TH_WH + tid, accWh);
  if (tid == 0) atomicAdd(grad + TH_BH, accBh);
}

// ---------------------------------------------------------------- parameters
// Packed copy of parameter i: BF16 for the convolution weights, FP32 for the
// biases and the head.
__device__ __forceinline__ void pack_one(unsigned char* packed, int i, float w) {
  if (i < TH_B1) {
    reinterpret_cast<__nv_bfloat16*>(packed + PK_W1)[i] = __float2bfloat16_rn(w);
  } else if (i < TH_W2) {
    reinterpret_cast<float*>(packed + PK_F32)[i - TH_B1] = w;
  } else if (i < TH_B2) {
    reinterpret_cast<__nv_bfloat16*>(packed + PK_W2)[i - TH_W2] = __float2bfloat16_rn(w);
  } else if (i < TH_W3) {
    reinterpret_cast<float*>(packed + PK_F32)[CH + i - TH_B2] = w;
  } else if (i < TH_B3) {
    reinterpret_cast<__nv_bfloat16*>(packed + PK_W3)[i - TH_W3] = __float2bfloat16_rn(w);
  } else {
    reinterpret_cast<float*>(packed + PK_F32)[2 * CH + i - TH_B3] = w;  // b3, wh, bh
  }
}

__global__ void k_cnn_pack(const float* __restrict__ theta, unsigned char* __restrict__ packed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N_PARAMS) pack_one(packed, i, theta[i]);
}

// Adam with bias correction (c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t));
// the gradient is consumed (zeroed) and the packed copy refreshed.
__global__ void k_cnn_adam(float* __restrict__ theta, float* __restrict__ m,
                           float* __restrict__ v, float* __restrict__ grad,
                           unsigned char* __restrict__ packed, AdamConsts k) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N_PARAMS) return;
  const float g = grad[i];
  const float mi = fmaf(k.beta1, m[i], k.one_minus_beta1 * g);
  const float vi = fmaf(k.beta2, v[i], k.one_minus_beta2 * g * g);
  const float lr = k.lr, eps = k.eps, c1 = k.c1, c2 = k.c2;
  const float w = theta[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  m[i] = mi;
  v[i] = vi;
  theta[i] = w;
  grad[i] = 0.f;
  pack_one(packed, i, w);
}

// ---------------------------------------------------------------- decisions
__device__ __forceinline__ void set_box(LatBox& L, const int lo[3], const int step[3],
                                        const int cnt[3], const int tdim[3]) {
  for (int a = 0; a < 3; ++a) {
    L.lo[a] = lo[a];
    L.step[a] = step[a];
    L.cnt[a] = cnt[a];
  }
  L.tiles = lattice_tiles(cnt, tdim);
}

__device__ __forceinline__ void empty_box(LatBox& L) {
  for (int a = 0; a < 3; ++a) {
    L.lo[a] = 0;
    L.step[a] = 1;
    L.cnt[a] = 0;
  }
  L.tiles = 0;
}

// One thread per scan. Level `level` of the proposal has scored the map of
// the scan's current region: descend into the proposed segment, or hand the
// scan to the Eq. 5 framework (its decimated profile box) when the softmax
// confidence is below the threshold.
__global__ void k_learned_decide(const LearnParams P, int level) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.B) return;
  LearnState st = P.state[s];
  uwb_result* R = P.out + s;
  if (level == 0) {
    st.lo[0] = st.lo[1] = 0;
    st.side = P.n;
    st.fallback = 0;
    st.map_points = 0;
    P.learned[s] = 0;
    empty_box(P.prof_boxes[s]);
  }
  if (st.fallback) {
    empty_box(P.map_boxes[s]);
    P.state[s] = st;
    return;
  }
  st.map_points += MAP * MAP;
  const float* z = P.scores + static_cast<size_t>(s) * SEGS;
  int best = 0;
  float zmax = z[0];
  for (int k = 1; k < SEGS; ++k)
    if (z[k] > zmax) {  // the first maximum wins ties
      zmax = z[k];
      best = k;
    }
  float sum = 0.f, second = 0.f;
  for (int k = 0; k < SEGS; ++k) {
    const float e = expf(z[k] - zmax);
    sum += e;
    if (k != best) second = fmaxf(second, e);
  }
  const float conf = 1.0f / sum;  // softmax probability of the best segment
  R->child[level] = best;
  R->n_children[level] = SEGS;
  R->metric_top[level] = conf;
  R->metric_gap[level] = 1.0 - static_cast<double>(second);
  R->n_logged = level + 1;
  if (!(conf >= P.threshold)) {
    st.fallback = 1;
    empty_box(P.map_boxes[s]);
    P.learned[s] = 0;
    const int step[3] = {P.dstep[0], P.dstep[1], P.dstep[2]};
    set_box(P.prof_boxes[s], P.doff, step, P.dcnt, P.tdim_final);
  } else {
    const int sub = st.side / SEG;
    st.lo[0] += (best % SEG) * sub;
    st.lo[1] += (best / SEG) * sub;
    st.side = sub;
    R->box_lo[level][0] = st.lo[0];
    R->box_lo[level][1] = st.lo[1];
    R->box_hi[level][0] = st.lo[0] + sub;
    R->box_hi[level][1] = st.lo[1] + sub;
    R->box_hi[level][2] = 1;
    R->iters = level + 1;
    if (level + 1 < P.levels) {
      const int step = sub / MAP, o = (step - 1) / 2;
      const int lo[3] = {st.lo[0] + o, st.lo[1] + o, 0};
      const int stp[3] = {step, step, 1};
      const int cnt[3] = {MAP, MAP, 1};
      set_box(P.map_boxes[s], lo, stp, cnt, P.tdim_map);
    } else {
      // final region: the segment framed by ceil(num / den * side) points per side
      const int fr = (P.frame_num * sub + P.frame_den - 1) / P.frame_den;
      int lo[3], cnt[3];
      const int stp[3] = {1, 1, 1};
      for (int a = 0; a < 2; ++a) {
        lo[a] = max(st.lo[a] - fr, 0);
        cnt[a] = min(st.lo[a] + sub + fr, P.n) - lo[a];
      }
      lo[2] = 0;
      cnt[2] = 1;
      set_box(P.final_boxes[s], lo, stp, cnt, P.tdim_final);
      empty_box(P.map_boxes[s]);
      P.learned[s] = 1;
      R->status = UWB_OK;
      R->stop_reason = UWB_STOP_LEARNED;
      for (int a = 0; a < 3; ++a) {
        R->roi_lo[a] = lo[a];
        R->roi_hi[a] = lo[a] + cnt[a];
        R->loc_idx[a] = -1;
      }
    }
  }
  P.state[s] = st;
}

// Coarse-map lattice of scan s's square region [lo, lo + side)^2 (region_lo
// [B][2] = (x, y)); regions outside the grid are recorded and left empty.
__global__ void k_region_boxes(const int* region_lo, int side, int n, int B, int tx, int ty,
                               LatBox* boxes, int* status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  const int x0 = region_lo[2 * s], y0 = region_lo[2 * s + 1];
  const int step = side / MAP, o = (step - 1) / 2;
  const int tdim[3] = {tx, ty, 1};
  if (x0 < 0 || y0 < 0 || x0 + side > n || y0 + side > n) {
    if (status) atomicExch(status, UWB_ERR_ARG);
    empty_box(boxes[s]);
    return;
  }
  const int lo[3] = {x0 + o, y0 + o, 0}, stp[3] = {step, step, 1}, cnt[3] = {MAP, MAP, 1};
  set_box(boxes[s], lo, stp, cnt, tdim);
}

}  // namespace

cudaError_t launch_region_boxes(const int* region_lo, int side, int n, int B, const int tdim[3],
                                LatBox* boxes, int* status, cudaStream_t st) {
  k_region_boxes<<<(B + 127) / 128, 128, 0, st>>>(region_lo, side, n, B, tdim[0], tdim[1], boxes,
                                                  status);
  return cudaGetLastError();
}

// The dynamic shared-memory limit of a kernel, raised once per device.
static bool smem_ready(const void* fn, int smem, int* done) {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return false;
  if (done[d]) return true;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return false;
  done[d] = 1;  // a race only repeats the same call
  return true;
}
static int g_fwd_attr[64], g_bwd_attr[64], g_self_attr[64];

size_t forward_smem() { return F_SMEM; }
size_t backward_smem() { return G_SMEM; }
size_t selftest_smem() { return ST_SMEM; }

cudaError_t launch_selftest(const uint16_t* a, const uint16_t* b, float* d, int* status,
                            cudaStream_t st) {
  if (!smem_ready(reinterpret_cast<const void*>(k_umma_selftest), ST_SMEM, g_self_attr))
    return cudaErrorInvalidValue;
  k_umma_selftest<<<1, 128, ST_SMEM, st>>>(a, b, d, status);
  return cudaGetLastError();
}

cudaError_t launch_forward(const void* packed, const float* maps, int B, float* scores,
                           const int* labels, void* save, float* loss, int* status, int ctas,
                           cudaStream_t st) {
  if (!smem_ready(reinterpret_cast<const void*>(k_cnn_forward), F_SMEM, g_fwd_attr))
    return cudaErrorInvalidValue;
  k_cnn_forward<<<ctas, F_THREADS, F_SMEM, st>>>(static_cast<const unsigned char*>(packed), maps, B,
                                               scores, labels, static_cast<unsigned char*>(save),
                                               loss, status);
  return cudaGetLastError();
}

cudaError_t launch_backward(const void* packed, void* save, int B, float* grad, int ctas,
                            cudaStream_t st) {
  if (!smem_ready(reinterpret_cast<const void*>(k_cnn_backward), G_SMEM, g_bwd_attr))
    return cudaErrorInvalidValue;
  k_cnn_backward<<<ctas, THREADS, G_SMEM, st>>>(static_cast<const unsigned char*>(packed),
                                                static_cast<unsigned char*>(save), B, grad);
  return cudaGetLastError();
}

cudaError_t launch_pack(const float* theta, void* packed, cudaStream_t st) {
  k_cnn_pack<<<(N_PARAMS + 255) / 256, 256, 0, st>>>(theta, static_cast<unsigned char*>(packed));
  return cudaGetLastError();
}

cudaError_t launch_adam(float* theta, float* m, float* v, float* grad, void* packed,
                        const AdamConsts& k, cudaStream_t st) {
  k_cnn_adam<<<(N_PARAMS + 255) / 256, 256, 0, st>>>(theta, m, v, grad,
                                                     static_cast<unsigned char*>(packed), k);
  return cudaGetLastError();
}

cudaError_t launch_decide(const LearnParams& p, int level, cudaStream_t st) {
  k_learned_decide<<<(p.B + 127) / 128, 128, 0, st>>>(p, level);
  return cudaGetLastError();
}

}  // namespace cnn
}  // namespace uwb
