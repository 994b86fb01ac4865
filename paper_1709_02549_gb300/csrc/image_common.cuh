// Confocal energy image over box lattices of the focal grid.
//
// Section II.A, Eq. 1 (delay, read as the round trip 2|r - a_i| / v in
// samples) and Eq. 3 (DAS: window sum of the squared antenna sum); Section
// II.B (DMAS: every pair of aligned signals multiplied and summed, then
// squared and window-summed like DAS).
//
// Execution model (one kernel for every lattice the method evaluates: the
// full grid, the decimated lattice, or one final region per scan):
//  * persistent CTAs, each owning a contiguous range of (scan, tile) work
//    items, so consecutive tiles of one scan reuse the staged traces;
//  * per scan, the window of samples any focal point of the lattice can read
//    (computed on the device from the antenna positions and the lattice's
//    bounding box) is copied to shared memory by one 3-D TMA box
//    (x = sample, y = antenna, z = scan) whose out-of-range elements arrive as
//    zeros -- exactly the "samples outside the trace are 0" convention;
//  * tiles of a lattice are linear (points in x-fastest order) or shaped
//    (tdim points per axis); one focal point per thread (two as float2 lanes
//    for uniform DAS and identity DMAS); the delay is computed in registers,
//    the W+1 samples of the window are read from shared memory and
//    interpolated;
//  * fused epilogue: image store, compact-profile store, and a 64-bit
//    (energy, -index) key per thread, reduced by the CTA once per scan and
//    folded into the scan's argmax with atomicMax.
// Scans whose window does not fit the staged span fall back to bounds-checked
// global loads (same arithmetic). Traces may be stored as float32, float16 or
// bfloat16; the staged window is always float32 (16-bit traces land in a raw
// area first and are widened once per staging), so the arithmetic is float32
// in every case.
#pragma once

#include <climits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ptx.cuh"
#include "uwb_internal.cuh"

namespace uwb {

// Bounded waits: a staging wait gives up after this many try_wait probes.
constexpr long kWaitProbes = 1L << 24;

// Antenna-to-focal-point distance with the hardware square-root
// approximation (sqrt.approx.f32, relative error about one float ulp): the
// IEEE-rounded sqrtf adds a branch and several instructions per antenna, and
// one ulp of distance is 1e-5 samples of delay at these scales, far below the
// image tolerance.
__device__ __forceinline__ float dist3(float dx, float dy, float dz) {
  const float q = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  float d;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(d) : "f"(q));
  return d;
}

// Launch shape of an instance. pp = focal points per thread: uniform
// monostatic DAS and identity DMAS evaluate two points per thread as the two
// lanes of paired (float2) instructions; a tile always holds threads * pp
// points. Multistatic and ragged (per-scan descriptor) instances keep one
// point per thread: their windows (up to 96 rows, or channel rows) often
// exceed the staged span, and on the global-load path 256 threads of one
// point measured faster than 128 of two.
template <int BF, int V, bool MS, bool RG>
struct KernelShape {
  static constexpr bool lit = BF == BF_DMAS_LIT;
  static constexpr bool pair = !lit && !RG;
  static constexpr int pp = pair ? 2 : 1;
  static constexpr int threads = (lit || (pair && !MS)) ? 128 : 256;
  // literal DMAS: 4 resident CTAs (<= 128 registers) up to 32 antennas, 2
  // for the 64-antenna block, 3 for the 96-antenna block form (no delay table).
  // Monostatic point pairs: DAS 4 and identity DMAS 3, where the paired
  // window accumulators fit registers (twice as many when the host launches
  // them with 64 threads, for few trace rows); ragged (one point per thread): DAS 3,
  // identity DMAS 2. Multistatic: one CTA per SM (its channel window takes
  // most of the shared memory), 256 threads of two points.
  static constexpr int min_blocks =
      lit ? (V <= 32 ? 4 : (V <= 64 ? 2 : 3))
          : (MS ? 1 : (pair ? (BF == BF_DAS ? 4 : 3) : (BF == BF_DAS ? 3 : 2)));
};

// Per-scan quantities: ragged instances (RG) read the scan's descriptor in
// shared memory; uniform instances read the launch parameters, which stay
// operands of the instructions that use them rather than occupying registers.
template <bool RG>
__device__ __forceinline__ int scan_M(const ImgParams& P, const ScanDesc* sS) {
  return RG ? sS->M : P.M;
}
template <bool RG>
__device__ __forceinline__ int scan_R(const ImgParams& P, const ScanDesc* sS) {
  return RG ? sS->R : P.R;
}
template <bool RG>
__device__ __forceinline__ float scan_kscale(const ImgParams& P, const ScanDesc* sS) {
  return RG ? sS->kscale : P.kscale;
}
template <bool RG>
__device__ __forceinline__ float scan_org(const ImgParams& P, const ScanDesc* sS, int a) {
  return RG ? sS->org[a] : P.org[a];
}
template <bool RG>
__device__ __forceinline__ float scan_pit(const ImgParams& P, const ScanDesc* sS, int a) {
  return RG ? sS->pit[a] : P.pit[a];
}
template <bool RG>
__device__ __forceinline__ int scan_gn(const ImgParams& P, const ScanDesc* sS, int a) {
  return RG ? sS->gn[a] : P.gn[a];
}

// One stored sample, widened to float32 (global-load path).
__device__ __forceinline__ float ld_trace(const void* base, long long i, int dtype) {
  if (dtype == DT_F32) return __ldg(static_cast<const float*>(base) + i);
  const unsigned short b = __ldg(static_cast<const unsigned short*>(base) + i);
  return dtype == DT_F16 ? __half2float(__ushort_as_half(b))
                         : __bfloat162float(__ushort_as_bfloat16(b));
}

// Sample n (absolute index) of trace row i, zero outside the stored range.
__device__ __forceinline__ float sample_at(const ScanDesc& S, int dtype, int i, int n) {
  const int o = n - S.n_begin;
  if (o < 0 || o >= S.N) return 0.f;
  return ld_trace(S.traces, static_cast<long long>(i) * S.pitch + o, dtype);
}

// Bounds-checked builds (nvcc -DUWB_CHECK, the library's stand-in for a
// memory checker): the first index of every run of `count` elements a kernel
// is about to read or write in a buffer of n elements is checked; a run that
// leaves the buffer records UWB_ERR_BOUNDS in the status word and is moved
// to index 0, so the access stays inside the buffer. Other builds return the
// index unchanged, and the checks compile away.
__device__ __forceinline__ int check_run(int* status, int first, int count, int n) {
#ifdef UWB_CHECK
  if (first < 0 || first > n - count) {
    atomicExch(status, UWB_ERR_BOUNDS);
    return 0;
  }
#endif
  return first;
}
__device__ __forceinline__ long long check_run64(int* status, long long first, long long n) {
#ifdef UWB_CHECK
  if (first < 0 || first >= n) {
    atomicExch(status, UWB_ERR_BOUNDS);
    return 0;
  }
#endif
  return first;
}

// -------------------------------------------------------------- DAS / DMAS-identity
// Rows are the M antennas (monostatic: delay 2|r - a_i| fs / v) or, with MS,
// the R channels (transmitter, receiver) of a multistatic recording (Eq. 2:
// delay (|r - a_tx| + |r - a_rx|) fs / v); for MS each thread first puts its
// focal point's distance to every antenna in sD[antenna][thread].
template <int BF, int WT, bool STAGED, bool MS, bool RG>
__device__ __forceinline__ float energy_sum(const ImgParams& P, const ScanDesc* __restrict__ sS,
                                            const float* __restrict__ sTr,
                                            const float4* __restrict__ sAnt,
                                            const int2* __restrict__ sCh, float* __restrict__ sD,
                                            int nlo, int cl_lo, int cl_hi, float px, float py,
                                            float pz) {
  float energy = 0.f;
  const int R = scan_R<RG>(P, sS);
  const float kscale = scan_kscale<RG>(P, sS);
  const int T = blockDim.x, tid = threadIdx.x;
  if (MS) {
    const int M = scan_M<RG>(P, sS);
    for (int i = 0; i < M; ++i) {
      const float4 a = sAnt[i];
      const float dx = px - a.x, dy = py - a.y, dz = pz - a.z;
      sD[i * T + tid] = dist3(dx, dy, dz);
    }
  }
  const float half_k = 0.5f * kscale;
  for (int k0 = 0; k0 < P.W; k0 += WT) {
    float s1[WT], s2[WT];
#pragma unroll
    for (int k = 0; k < WT; ++k) {
      s1[k] = 0.f;
      s2[k] = 0.f;
    }
    const float hoff = static_cast<float>(P.h - k0);
    for (int i = 0; i < R; ++i) {
      float t;  // u_i - h + k0
      if (MS) {
        const int2 c = sCh[i];
        t = fmaf(sD[c.x * T + tid] + sD[c.y * T + tid], half_k, -hoff);
      } else {
        const float4 a = sAnt[i];
        const float dx = px - a.x;
        const float dy = py - a.y;
        const float dz = pz - a.z;
        const float d = dist3(dx, dy, dz);
        t = fmaf(d, kscale, -hoff);
      }
      const float fl = floorf(t);
      const float f = t - fl;
      int n0 = static_cast<int>(fl);
      float y[WT + 1];
      if (STAGED) {
        n0 = min(max(n0, cl_lo), cl_hi);
        const float* row =
            sTr + check_run(P.status, i * P.span + (n0 - nlo), WT + 1, P.Rcap * P.span);
#pragma unroll
        for (int k = 0; k <= WT; ++k) y[k] = row[k];
      } else {
        const ScanDesc S = *sS;
#pragma unroll
        for (int k = 0; k <= WT; ++k) y[k] = sample_at(S, P.dtype, i, n0 + k);
      }
      if (BF == BF_DAS) {
        const float g = 1.f - f;
#pragma unroll
        for (int k = 0; k < WT; ++k) {
          s1[k] = fmaf(g, y[k], s1[k]);
          s1[k] = fmaf(f, y[k + 1], s1[k]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < WT; ++k) {
          const float x = fmaf(f, y[k + 1] - y[k], y[k]);
          s1[k] += x;
          s2[k] = fmaf(x, x, s2[k]);
        }
      }
    }
    const int kend = min(WT, P.W - k0);
#pragma unroll
    for (int k = 0; k < WT; ++k) {
      if (k < kend) {
        if (BF == BF_DAS) {
          energy = fmaf(s1[k], s1[k], energy);
        } else {
          // sum_{i<j} x_i x_j; the square is rounded like s2's terms (no fused
          // multiply-add) so a single antenna gives exactly zero
          const float p = 0.5f * (__fmul_rn(s1[k], s1[k]) - s2[k]);
          energy = fmaf(p, p, energy);
        }
      }
    }
  }
  return energy;
}

// Two focal points per thread (monostatic rows, staged window): the lanes of
// every float2 are the two points, so each per-sample multiply-add of the
// window sums is half of one paired instruction. Lane by lane the operations
// and their order are those of energy_sum (a - b is formed as the fused
// b * (-1) + a, which rounds the same), so both give identical energies.
template <int BF, int WT, bool RG, bool MS>
__device__ __forceinline__ float2 energy_sum_pair(const ImgParams& P,
                                                  const ScanDesc* __restrict__ sS,
                                                  const float* __restrict__ sTr,
                                                  const float4* __restrict__ sAnt,
                                                  const int2* __restrict__ sCh,
                                                  float* __restrict__ sD, int nlo, int cl_lo,
                                                  int cl_hi, float2 px, float2 py, float2 pz) {
  const float2 one = make_float2(1.f, 1.f), m1 = make_float2(-1.f, -1.f);
  float2 energy = make_float2(0.f, 0.f);
  const int R = scan_R<RG>(P, sS);
  const float kscale = scan_kscale<RG>(P, sS);
  const float2 ks = make_float2(kscale, kscale);
  // multistatic: the distance of each of this thread's two points to every
  // antenna, in sD[antenna][point of the CTA] (points v0 and v0 + blockDim)
  const int TP = 2 * blockDim.x, v0 = threadIdx.x, v1 = threadIdx.x + blockDim.x;
  if (MS) {
    const int M = scan_M<RG>(P, sS);
    for (int i = 0; i < M; ++i) {
      const float4 a = sAnt[i];
      const float2 dx = make_float2(px.x - a.x, px.y - a.x);
      const float2 dy = make_float2(py.x - a.y, py.y - a.y);
      const float2 dz = make_float2(pz.x - a.z, pz.y - a.z);
      const float2 q = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
      float dxv, dyv;
      asm("sqrt.approx.f32 %0, %1;" : "=f"(dxv) : "f"(q.x));
      asm("sqrt.approx.f32 %0, %1;" : "=f"(dyv) : "f"(q.y));
      sD[i * TP + v0] = dxv;
      sD[i * TP + v1] = dyv;
    }
  }
  const float half_k = 0.5f * kscale;
  for (int k0 = 0; k0 < P.W; k0 += WT) {
    float2 s1[WT], s2[WT];
#pragma unroll
    for (int k = 0; k < WT; ++k) {
      s1[k] = make_float2(0.f, 0.f);
      s2[k] = make_float2(0.f, 0.f);
    }
    const float hoff = static_cast<float>(P.h - k0);
    const float2 nh = make_float2(-hoff, -hoff);
    for (int i = 0; i < R; ++i) {
      float2 t;  // u_i - h + k0 for both points
      if (MS) {
        // Eq. 2: (|r - a_tx| + |r - a_rx|) fs / v, lane by lane as energy_sum
        const int2 c = sCh[i];
        t.x = fmaf(sD[c.x * TP + v0] + sD[c.y * TP + v0], half_k, -hoff);
        t.y = fmaf(sD[c.x * TP + v1] + sD[c.y * TP + v1], half_k, -hoff);
      } else {
        const float4 a = sAnt[i];
        const float2 dx = make_float2(px.x - a.x, px.y - a.x);
        const float2 dy = make_float2(py.x - a.y, py.y - a.y);
        const float2 dz = make_float2(pz.x - a.z, pz.y - a.z);
        // dist3 lane by lane: dx^2 + (dy^2 + dz^2), then the approximate root
        const float2 q = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
        float2 d;
        asm("sqrt.approx.f32 %0, %1;" : "=f"(d.x) : "f"(q.x));
        asm("sqrt.approx.f32 %0, %1;" : "=f"(d.y) : "f"(q.y));
        t = __ffma2_rn(d, ks, nh);
      }
      const float2 fl = make_float2(floorf(t.x), floorf(t.y));
      const float2 f = __ffma2_rn(fl, m1, t);
      const int nx = min(max(static_cast<int>(fl.x), cl_lo), cl_hi);
      const int ny = min(max(static_cast<int>(fl.y), cl_lo), cl_hi);
      const float* rx =
          sTr + check_run(P.status, i * P.span + (nx - nlo), WT + 1, P.Rcap * P.span);
      const float* ry =
          sTr + check_run(P.status, i * P.span + (ny - nlo), WT + 1, P.Rcap * P.span);
      float2 y[WT + 1];
#pragma unroll
      for (int k = 0; k <= WT; ++k) y[k] = make_float2(rx[k], ry[k]);
      if (BF == BF_DAS) {
        const float2 g = __ffma2_rn(f, m1, one);
#pragma unroll
        for (int k = 0; k < WT; ++k) {
          s1[k] = __ffma2_rn(g, y[k], s1[k]);
          s1[k] = __ffma2_rn(f, y[k + 1], s1[k]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < WT; ++k) {
          const float2 x = __ffma2_rn(f, __ffma2_rn(y[k], m1, y[k + 1]), y[k]);
          s1[k] = __fadd2_rn(s1[k], x);
          s2[k] = __ffma2_rn(x, x, s2[k]);
        }
      }
    }
    const int kend = min(WT, P.W - k0);
#pragma unroll
    for (int k = 0; k < WT; ++k) {
      if (k < kend) {
        if (BF == BF_DAS) {
          energy = __ffma2_rn(s1[k], s1[k], energy);
        } else {
          const float2 sq = __fmul2_rn(s1[k], s1[k]);
          const float2 p = __fmul2_rn(make_float2(0.5f, 0.5f), __ffma2_rn(s2[k], m1, sq));
          energy = __ffma2_rn(p, p, energy);
        }
      }
    }
  }
  return energy;
}

// ------------------------------------------------------------------ literal DMAS
// Two window samples (k, k+1) travel together as a float2, so every antenna
// pair costs one paired FMA for both samples. The pair sum
// sum_{i<j} x_i x_j forms every product explicitly (MMAX(MMAX-1)/2 paired
// FMAs over eight accumulators), streaming over j: antenna j is interpolated
// and immediately multiplied with antennas 0..j-1, while the samples of
// antenna j+1 are already being loaded. Antenna slots beyond M read zero rows
// of shared memory (or zeros on the global path) and add nothing.

// Raw inputs of one antenna's interpolation for one window pair.
struct LitRaw {
  float f, y0, y1, y2;
};

template <bool STAGED, bool RG>
__device__ __forceinline__ LitRaw lit_load(const ImgParams& P, const ScanDesc* __restrict__ sS,
                                           const float* __restrict__ sTr,
                                           const float2* __restrict__ sNF, int i, int T, int tid,
                                           int k0) {
  const float2 nf = sNF[i * T + tid];
  const int off = __float_as_int(nf.x) + k0;
  LitRaw r;
  r.f = nf.y;
  if (STAGED) {
    // nf.x holds the shared-window byte address of sample 0 of this antenna's
    // window: three loads at immediate offsets, no per-antenna address scaling
    const uint32_t a = __float_as_uint(nf.x) + 4u * static_cast<uint32_t>(k0);
    asm volatile(
        "ld.shared.f32 %0, [%3];\n\t"
        "ld.shared.f32 %1, [%3+4];\n\t"
        "ld.shared.f32 %2, [%3+8];"
        : "=f"(r.y0), "=f"(r.y1), "=f"(r.y2)
        : "r"(a));
  } else if (i < scan_M<RG>(P, sS)) {
    const ScanDesc S = *sS;
    r.y0 = sample_at(S, P.dtype, i, off);
    r.y1 = sample_at(S, P.dtype, i, off + 1);
    r.y2 = sample_at(S, P.dtype, i, off + 2);
  } else {
    r.y0 = r.y1 = r.y2 = 0.f;
  }
  return r;
}

// x(k) = (1 - f) y[n0+k] + f y[n0+k+1] for the two samples of the pair
__device__ __forceinline__ float2 lit_interp(const LitRaw& r) {
  const float2 lo = make_float2(r.y0, r.y1);
  const float2 t = __ffma2_rn(make_float2(-r.f, -r.f), lo, lo);
  return __ffma2_rn(make_float2(r.f, r.f), make_float2(r.y1, r.y2), t);
}

// sTr holds MMAX rows; rows M..MMAX-1 are zero (written at each staging).
template <int MMAX, bool STAGED, bool RG>
__device__ __forceinline__ float energy_literal(const ImgParams& P,
                                                const ScanDesc* __restrict__ sS,
                                                const float* __restrict__ sTr,
                                                const float4* __restrict__ sAnt,
                                                float2* __restrict__ sNF, int nlo, int cl_lo,
                                                int cl_hi, float px, float py, float pz) {
  // the literal kernel always runs 128 threads: a constant T turns the
  // per-antenna (offset, fraction) addresses into immediate offsets
  constexpr int T = KernelShape<BF_DMAS_LIT, MMAX, false, false>::threads;
  const int tid = threadIdx.x;
  const int M = scan_M<RG>(P, sS);
  const float kscale = scan_kscale<RG>(P, sS);
  const float hf = static_cast<float>(P.h);
  // delays of every antenna for this focal point: (sample offset, fraction)
  for (int i = 0; i < MMAX; ++i) {
    int n0 = 0;
    float f = 0.f;
    if (i < M) {
      const float4 a = sAnt[i];
      const float dx = px - a.x;
      const float dy = py - a.y;
      const float dz = pz - a.z;
      const float d = dist3(dx, dy, dz);
      const float t = fmaf(d, kscale, -hf);
      const float fl = floorf(t);
      f = t - fl;
      n0 = static_cast<int>(fl);
      // the passes read the words [first, first + wpad] of the row
      if (STAGED)
        n0 = static_cast<int>(smem_u32(sTr)) +
             4 * check_run(P.status, min(max(n0, cl_lo), cl_hi) - nlo + i * P.span, P.wpad + 1,
                           MMAX * P.span);
    } else if (STAGED) {
      // rows M..MMAX-1 of the staged window are zero
      n0 = static_cast<int>(smem_u32(sTr)) + 4 * i * P.span;
    }
    sNF[i * T + tid] = make_float2(__int_as_float(n0), f);
  }
  float energy = 0.f;
  for (int k0 = 0; k0 < P.W; k0 += 2) {
    float2 x[MMAX];
    float2 acc[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) acc[a] = make_float2(0.f, 0.f);
    LitRaw next = lit_load<STAGED, RG>(P, sS, sTr, sNF, 0, T, tid, k0);
#pragma unroll
    for (int j = 0; j < MMAX; ++j) {
      const LitRaw cur = next;
      if (j + 1 < MMAX) next = lit_load<STAGED, RG>(P, sS, sTr, sNF, j + 1, T, tid, k0);
      x[j] = lit_interp(cur);
#pragma unroll
      for (int i = 0; i < j; ++i) acc[(i + j) & 7] = __ffma2_rn(x[i], x[j], acc[(i + j) & 7]);
      // keep later loads from being hoisted above these products
      asm volatile("" ::: "memory");
    }
    const float2 s01 = __fadd2_rn(acc[0], acc[1]), s23 = __fadd2_rn(acc[2], acc[3]);
    const float2 s45 = __fadd2_rn(acc[4], acc[5]), s67 = __fadd2_rn(acc[6], acc[7]);
    const float2 p = __fadd2_rn(__fadd2_rn(s01, s23), __fadd2_rn(s45, s67));
    energy = fmaf(p.x, p.x, energy);
    if (k0 + 1 < P.W) energy = fmaf(p.y, p.y, energy);
  }
  return energy;
}

// Four window samples per pass (k0 .. k0 + 3) as two float2 streams: the
// per-antenna loads, offset and interpolation work is shared by twice as many
// pair products as in energy_literal. Used for the 16-antenna register block,
// where the 2 x 16 float2 values still allow 4 resident CTAs; for 32 antennas
// the pair version at 4 CTAs per SM measured faster than this one at 2.
struct LitRaw4 {
  float y0, y1, y2, y3, y4, f;
};

template <bool STAGED, bool RG>
__device__ __forceinline__ LitRaw4 lit_load4(const ImgParams& P, const ScanDesc* __restrict__ sS,
                                             const float* __restrict__ sTr,
                                             const float2* __restrict__ sNF, int i, int T,
                                             int tid, int k0) {
  const float2 nf = sNF[i * T + tid];
  const int off = __float_as_int(nf.x) + k0;
  LitRaw4 r;
  r.f = nf.y;
  if (STAGED) {  // nf.x: shared-window byte address of the antenna's window (see lit_load)
    const uint32_t a = __float_as_uint(nf.x) + 4u * static_cast<uint32_t>(k0);
    asm volatile(
        "ld.shared.f32 %0, [%5];\n\t"
        "ld.shared.f32 %1, [%5+4];\n\t"
        "ld.shared.f32 %2, [%5+8];\n\t"
        "ld.shared.f32 %3, [%5+12];\n\t"
        "ld.shared.f32 %4, [%5+16];"
        : "=f"(r.y0), "=f"(r.y1), "=f"(r.y2), "=f"(r.y3), "=f"(r.y4)
        : "r"(a));
  } else if (i < scan_M<RG>(P, sS)) {
    const ScanDesc S = *sS;
    r.y0 = sample_at(S, P.dtype, i, off);
    r.y1 = sample_at(S, P.dtype, i, off + 1);
    r.y2 = sample_at(S, P.dtype, i, off + 2);
    r.y3 = sample_at(S, P.dtype, i, off + 3);
    r.y4 = sample_at(S, P.dtype, i, off + 4);
  } else {
    r.y0 = r.y1 = r.y2 = r.y3 = r.y4 = 0.f;
  }
  return r;
}

template <int MMAX, bool STAGED, bool RG>
__device__ __forceinline__ float energy_literal4(const ImgParams& P,
                                                 const ScanDesc* __restrict__ sS,
                                                 const float* __restrict__ sTr,
                                                 const float4* __restrict__ sAnt,
                                                 float2* __restrict__ sNF, int nlo, int cl_lo,
                                                 int cl_hi, float px, float py, float pz) {
  // the literal kernel always runs 128 threads: a constant T turns the
  // per-antenna (offset, fraction) addresses into immediate offsets
  constexpr int T = KernelShape<BF_DMAS_LIT, MMAX, false, false>::threads;
  const int tid = threadIdx.x;
  const int M = scan_M<RG>(P, sS);
  const float kscale = scan_kscale<RG>(P, sS);
  const float hf = static_cast<float>(P.h);
  for (int i = 0; i < MMAX; ++i) {
    int n0 = 0;
    float f = 0.f;
    if (i < M) {
      const float4 a = sAnt[i];
      const float dx = px - a.x;
      const float dy = py - a.y;
      const float dz = pz - a.z;
      const float d = dist3(dx, dy, dz);
      const float t = fmaf(d, kscale, -hf);
      const float fl = floorf(t);
      f = t - fl;
      n0 = static_cast<int>(fl);
      // the passes read the words [first, first + wpad] of the row
      if (STAGED)
        n0 = static_cast<int>(smem_u32(sTr)) +
             4 * check_run(P.status, min(max(n0, cl_lo), cl_hi) - nlo + i * P.span, P.wpad + 1,
                           MMAX * P.span);
    } else if (STAGED) {
      // rows M..MMAX-1 of the staged window are zero
      n0 = static_cast<int>(smem_u32(sTr)) + 4 * i * P.span;
    }
    sNF[i * T + tid] = make_float2(__int_as_float(n0), f);
  }
  float energy = 0.f;
  for (int k0 = 0; k0 < P.W; k0 += 4) {
    float2 xa[MMAX], xb[MMAX];
    float2 acc[8], bcc[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      acc[a] = make_float2(0.f, 0.f);
      bcc[a] = make_float2(0.f, 0.f);
    }
    LitRaw4 next = lit_load4<STAGED, RG>(P, sS, sTr, sNF, 0, T, tid, k0);
#pragma unroll
    for (int j = 0; j < MMAX; ++j) {
      const LitRaw4 cur = next;
      if (j + 1 < MMAX) next = lit_load4<STAGED, RG>(P, sS, sTr, sNF, j + 1, T, tid, k0);
      const float2 ff = make_float2(cur.f, cur.f), nf2 = make_float2(-cur.f, -cur.f);
      const float2 lo_a = make_float2(cur.y0, cur.y1), hi_a = make_float2(cur.y1, cur.y2);
      const float2 lo_b = make_float2(cur.y2, cur.y3), hi_b = make_float2(cur.y3, cur.y4);
      xa[j] = __ffma2_rn(ff, hi_a, __ffma2_rn(nf2, lo_a, lo_a));
      xb[j] = __ffma2_rn(ff, hi_b, __ffma2_rn(nf2, lo_b, lo_b));
#pragma unroll
      for (int i = 0; i < j; ++i) {
        acc[(i + j) & 7] = __ffma2_rn(xa[i], xa[j], acc[(i + j) & 7]);
        bcc[(i + j) & 7] = __ffma2_rn(xb[i], xb[j], bcc[(i + j) & 7]);
      }
      // keep later loads from being hoisted above these products
      asm volatile("" ::: "memory");
    }
    const float2 pa = __fadd2_rn(__fadd2_rn(__fadd2_rn(acc[0], acc[1]), __fadd2_rn(acc[2], acc[3])),
                                 __fadd2_rn(__fadd2_rn(acc[4], acc[5]), __fadd2_rn(acc[6], acc[7])));
    const float2 pb = __fadd2_rn(__fadd2_rn(__fadd2_rn(bcc[0], bcc[1]), __fadd2_rn(bcc[2], bcc[3])),
                                 __fadd2_rn(__fadd2_rn(bcc[4], bcc[5]), __fadd2_rn(bcc[6], bcc[7])));
    energy = fmaf(pa.x, pa.x, energy);
    if (k0 + 1 < P.W) energy = fmaf(pa.y, pa.y, energy);
    if (k0 + 2 < P.W) energy = fmaf(pb.x, pb.x, energy);
    if (k0 + 3 < P.W) energy = fmaf(pb.y, pb.y, energy);
  }
  return energy;
}

// ------------------------------------------------------- literal DMAS, blocks of 32
// Register blocks beyond 64 antennas (MMAX = 32 NB): for one window pair (k,
// k+1) the M(M-1)/2 products are formed block pair by block pair, every one
// explicitly. Block a's 32 interpolated sample pairs are held in registers
// while its own pairs are formed (a streamed triangle, as in energy_literal);
// then every antenna of each later block is interpolated and multiplied with
// the 32 held ones. A scan forms pairs only among its own M antennas. Each
// antenna's delay is recomputed at each visit: a per-thread (offset,
// fraction) table of 96 antennas would take 96 KB of shared memory per CTA
// beside the staged window, leaving one CTA per SM.

// Shared-window byte address (staged) or absolute sample index (global path)
// of sample 0 of antenna i's window for this focal point, and its fraction:
// the same arithmetic as energy_literal's table.
template <int ROWS, bool STAGED>
__device__ __forceinline__ int lit_delay(const ImgParams& P, const float4* __restrict__ sAnt,
                                         int i, float px, float py, float pz, float kscale,
                                         float hf, uint32_t base, int nlo, int cl_lo, int cl_hi,
                                         float& f) {
  const float4 a = sAnt[i];
  const float dx = px - a.x;
  const float dy = py - a.y;
  const float dz = pz - a.z;
  const float d = dist3(dx, dy, dz);
  const float t = fmaf(d, kscale, -hf);
  const float fl = floorf(t);
  f = t - fl;
  const int n0 = static_cast<int>(fl);
  // a window pair's passes read the words [first, first + wpad] of the row
  if (STAGED)
    return static_cast<int>(base) + 4 * check_run(P.status,
                                                  min(max(n0, cl_lo), cl_hi) - nlo + i * P.span,
                                                  P.wpad + 1, ROWS * P.span);
  return n0;
}

// The interpolated sample pair (k0, k0 + 1) of antenna i from its delay.
template <bool STAGED>
__device__ __forceinline__ float2 lit_pair(const ImgParams& P, const ScanDesc* __restrict__ sS,
                                           int i, int at, float f, int k0) {
  LitRaw r;
  r.f = f;
  if (STAGED) {
    const uint32_t a = static_cast<uint32_t>(at) + 4u * static_cast<uint32_t>(k0);
    asm volatile(
        "ld.shared.f32 %0, [%3];\n\t"
        "ld.shared.f32 %1, [%3+4];\n\t"
        "ld.shared.f32 %2, [%3+8];"
        : "=f"(r.y0), "=f"(r.y1), "=f"(r.y2)
        : "r"(a));
  } else {
    const ScanDesc S = *sS;
    r.y0 = sample_at(S, P.dtype, i, at + k0);
    r.y1 = sample_at(S, P.dtype, i, at + k0 + 1);
    r.y2 = sample_at(S, P.dtype, i, at + k0 + 2);
  }
  return lit_interp(r);
}

template <int NB, bool STAGED, bool RG>
__device__ __forceinline__ float energy_literal_blocks(const ImgParams& P,
                                                       const ScanDesc* __restrict__ sS,
                                                       const float* __restrict__ sTr,
                                                       const float4* __restrict__ sAnt, int nlo,
                                                       int cl_lo, int cl_hi, float px, float py,
                                                       float pz) {
  const int M = min(scan_M<RG>(P, sS), 32 * NB);
  const float kscale = scan_kscale<RG>(P, sS);
  const float hf = static_cast<float>(P.h);
  const uint32_t base = STAGED ? smem_u32(sTr) : 0u;
  const int nb = (M + 31) >> 5;
  float energy = 0.f;
  for (int k0 = 0; k0 < P.W; k0 += 2) {
    float2 acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int blk = 0; blk < nb; ++blk) {
      const int ia = 32 * blk;
      const int na = min(32, M - ia);
      // the held block: its own pairs, streamed one antenna ahead
      float2 xa[32];
      float fn;
      int an = lit_delay<32 * NB, STAGED>(P, sAnt, ia, px, py, pz, kscale, hf, base, nlo, cl_lo, cl_hi,
                                 fn);
      float2 xn = lit_pair<STAGED>(P, sS, ia, an, fn, k0);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        if (j < na) {
          const float2 x = xn;
          if (j + 1 < na) {
            an = lit_delay<32 * NB, STAGED>(P, sAnt, ia + j + 1, px, py, pz, kscale, hf, base, nlo, cl_lo,
                                   cl_hi, fn);
            xn = lit_pair<STAGED>(P, sS, ia + j + 1, an, fn, k0);
          }
#pragma unroll
          for (int i = 0; i < j; ++i) acc[(i + j) & 7] = __ffma2_rn(xa[i], x, acc[(i + j) & 7]);
          xa[j] = x;
        } else {
          xa[j] = make_float2(0.f, 0.f);
        }
        asm volatile("" ::: "memory");
      }
      // every antenna of the later blocks against the held block, four at a
      // time: the next four are interpolated (independent delay chains) while
      // the current four's 128 products run
      int jb = ia + 32;
      float2 xq[4];
      auto load4 = [&](int j0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float fq;
          const int aq = lit_delay<32 * NB, STAGED>(P, sAnt, j0 + q, px, py, pz, kscale, hf, base, nlo,
                                           cl_lo, cl_hi, fq);
          xq[q] = lit_pair<STAGED>(P, sS, j0 + q, aq, fq, k0);
        }
      };
      if (jb + 4 <= M) load4(jb);
#pragma unroll 1
      for (; jb + 4 <= M; jb += 4) {
        const float2 x0 = xq[0], x1 = xq[1], x2 = xq[2], x3 = xq[3];
        if (jb + 8 <= M) load4(jb + 4);
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i & 7] = __ffma2_rn(xa[i], x0, acc[i & 7]);
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i & 7] = __ffma2_rn(xa[i], x1, acc[i & 7]);
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i & 7] = __ffma2_rn(xa[i], x2, acc[i & 7]);
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i & 7] = __ffma2_rn(xa[i], x3, acc[i & 7]);
        asm volatile("" ::: "memory");
      }
#pragma unroll 1
      for (; jb < M; ++jb) {
        float fr;
        const int ar = lit_delay<32 * NB, STAGED>(P, sAnt, jb, px, py, pz, kscale, hf, base, nlo, cl_lo,
                                         cl_hi, fr);
        const float2 x = lit_pair<STAGED>(P, sS, jb, ar, fr, k0);
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i & 7] = __ffma2_rn(xa[i], x, acc[i & 7]);
      }
    }
    const float2 s01 = __fadd2_rn(acc[0], acc[1]), s23 = __fadd2_rn(acc[2], acc[3]);
    const float2 s45 = __fadd2_rn(acc[4], acc[5]), s67 = __fadd2_rn(acc[6], acc[7]);
    const float2 p = __fadd2_rn(__fadd2_rn(s01, s23), __fadd2_rn(s45, s67));
    energy = fmaf(p.x, p.x, energy);
    if (k0 + 1 < P.W) energy = fmaf(p.y, p.y, energy);
  }
  return energy;
}

template <int NB, bool RG>
__device__ __noinline__ float energy_literal_blocks_global(const ImgParams& P, const ScanDesc* sS,
                                                           const float4* sAnt, float px, float py,
                                                           float pz) {
  return energy_literal_blocks<NB, false, RG>(P, sS, nullptr, sAnt, 0, 0, 0, px, py, pz);
}

// The global-load fallback (a window wider than the staged span) runs as a
// real call, so its bounds checks and type conversions do not add to the
// register allocation of the staged hot path.
template <int BF, int WT, bool MS>
__device__ __noinline__ float energy_sum_global(const ImgParams& P, const ScanDesc* sS,
                                                const float4* sAnt, const int2* sCh, float* sD,
                                                float px, float py, float pz) {
  return energy_sum<BF, WT, false, MS, true>(P, sS, nullptr, sAnt, sCh, sD, 0, 0, 0, px, py, pz);
}

template <int MMAX>
__device__ __noinline__ float energy_literal_global(const ImgParams& P, const ScanDesc* sS,
                                                    const float4* sAnt, float2* sNF, float px,
                                                    float py, float pz) {
  if constexpr (MMAX <= 16)
    return energy_literal4<MMAX, false, true>(P, sS, nullptr, sAnt, sNF, 0, 0, 0, px, py, pz);
  else
    return energy_literal<MMAX, false, true>(P, sS, nullptr, sAnt, sNF, 0, 0, 0, px, py, pz);
}

// The descriptor of scan `scan`: from the per-scan array of a ragged batch, or
// derived from the uniform batch's parameters.
__device__ __forceinline__ void make_desc(const ImgParams& P, int scan, ScanDesc& S) {
  if (P.descs) {
    S = P.descs[scan];
    return;
  }
  S.traces = static_cast<const char*>(P.traces) +
             static_cast<long long>(scan) * P.trace_stride * dtype_bytes(P.dtype);
  S.ant = P.ant + static_cast<long long>(scan) * P.ant_stride;
  S.img_off = static_cast<long long>(scan) * P.gP;
  S.cmp_off = static_cast<long long>(scan) * P.compact_stride;
  S.pitch = P.pitch;
  S.n_begin = P.n_begin;
  S.N = P.N;
  S.M = P.M;
  S.R = P.R;
  S.tma = P.use_tma ? scan : -1;  // uniform: z coordinate of the launch's tensor map
  S.kscale = P.kscale;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    S.org[a] = P.org[a];
    S.pit[a] = P.pit[a];
    S.gn[a] = P.gn[a];
  }
}

// A CTA takes a dynamic share of the tiles only when the launch has at least
// this many per CTA; with fewer, a contiguous range stages fewer windows than
// chunks would. The 512 x 512 decimated profiles (5 tiles per CTA) measured
// 8 % faster with the counter than with contiguous ranges.
constexpr long long kDynMinTiles = 4;

// The scan that tile g of a ragged or boxed launch belongs to: the largest
// scan with prefix[scan] <= g (empty scans share their successor's prefix).
__device__ __forceinline__ int scan_of_tile(const ImgParams& P, long long g) {
  int lo = 0, hi = P.B;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (P.prefix[mid] <= g) lo = mid; else hi = mid;
  }
  return lo;
}

// ------------------------------------------------------------------ the kernel
// V = window chunk WT (DAS, DMAS identity) or antenna register block MMAX
// (literal DMAS); MS = multistatic rows. Dynamic shared memory as laid out by
// image_smem_layout.
template <int BF, int V, bool MS, bool RG>
__global__ void __launch_bounds__(KernelShape<BF, V, MS, RG>::threads,
                                   KernelShape<BF, V, MS, RG>::min_blocks)
    k_image(const __grid_constant__ CUtensorMap tmap, const ImgParams P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int T = blockDim.x, tid = threadIdx.x;
  // literal DMAS keeps V (>= M) trace rows; rows M..V-1 stay zero
  const int rows = (BF == BF_DMAS_LIT) ? V : P.Rcap;
  // per-point tables are sized by the CTA's focal points (threads x points per thread)
  const SmemLayout Lay = image_smem_layout(BF, P.Mcap, P.Rcap, rows, P.span,
                                           T * KernelShape<BF, V, MS, RG>::pp, MS, P.dtype);
  float* sTr = reinterpret_cast<float*>(smem_raw);
  unsigned short* sRaw = reinterpret_cast<unsigned short*>(smem_raw + Lay.raw);
  float4* sAnt = reinterpret_cast<float4*>(smem_raw + Lay.ant);  // (x, y, z, 0)
  int2* sCh = reinterpret_cast<int2*>(smem_raw + Lay.ch);
  float2* sNF = reinterpret_cast<float2*>(smem_raw + Lay.nf);
  float* sD = reinterpret_cast<float*>(smem_raw + Lay.d);
  ScanDesc* sS = reinterpret_cast<ScanDesc*>(smem_raw + Lay.desc);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + Lay.bar);
  unsigned long long* sKey = reinterpret_cast<unsigned long long*>(smem_raw + Lay.key);
  int* sInt = reinterpret_cast<int*>(smem_raw + Lay.ints);

  // point q of a thread is the tile's point number tid + q * T; shaped tiles
  // place it by warp sub-blocks of wdim points
  const int lane = tid & 31, warp = tid >> 5;
  constexpr int PP = KernelShape<BF, V, MS, RG>::pp;
  const bool linear = tile_linear(P.tdim);
  int lx[PP], ly[PP], lz[PP];
#pragma unroll
  for (int q = 0; q < PP; ++q) {
    lx[q] = ly[q] = lz[q] = 0;
    if (!linear) {
      const int nbx = P.tdim[0] / P.wdim[0], nby = P.tdim[1] / P.wdim[1];
      const int vw = warp + q * (T >> 5);
      lx[q] = (vw % nbx) * P.wdim[0] + lane % P.wdim[0];
      ly[q] = ((vw / nbx) % nby) * P.wdim[1] + (lane / P.wdim[0]) % P.wdim[1];
      lz[q] = (vw / (nbx * nby)) * P.wdim[2] + lane / (P.wdim[0] * P.wdim[1]);
    }
  }

  // where a TMA copy of the window lands: the float32 window itself, or the
  // raw 16-bit area that is widened afterwards
  void* tma_dst = P.dtype == DT_F32 ? static_cast<void*>(sTr) : static_cast<void*>(sRaw);
  const bool tma_ok = (P.use_tma || P.tmaps) && ((smem_u32(tma_dst) & 127u) == 0);
  if (tid == 0) mbar_init(bar, 1);
  if (MS) {
    // channel table (shared by every scan); indices outside the array are
    // recorded as an argument error and clamped so that no access leaves it
    const int M = P.M;
    for (int r = tid; r < P.R; r += T) {
      int2 c = P.chan[r];
      if (c.x < 0 || c.x >= M || c.y < 0 || c.y >= M) atomicExch(P.status, UWB_ERR_ARG);
      c.x = min(max(c.x, 0), M - 1);
      c.y = min(max(c.y, 0), M - 1);
      sCh[r] = c;
    }
  }
  __syncthreads();
  uint32_t phase = 0;

  const long long total =
      P.boxes ? static_cast<long long>(P.prefix[P.B]) : static_cast<long long>(P.B) * P.uni.tiles;
  // Work split. The CTAs that share an SM do not advance at equal rates: its
  // warp schedulers favour some of them. With equal contiguous ranges the
  // favoured CTAs finish early and the last one runs alone: on the 512 x 512
  // literal-DMAS final regions, the first CTA of every SM ended at 42 % of the
  // kernel's time and 2.9 of 4 CTAs were resident on average. With a tile
  // counter (P.work, zero at launch) and enough tiles per CTA, every CTA
  // instead takes chunks of consecutive tiles as it frees up. Chunks shrink
  // with the work left (guided self-scheduling: an eighth of an even share
  // of it, at least 2 tiles), so scans are rarely staged twice and the CTAs
  // end within a chunk of each other.
  const bool dyn = P.work != nullptr && total >= kDynMinTiles * static_cast<long long>(gridDim.x);
  long long g_begin = 0, g_end = 0;
  if (!dyn) {
    const long long chunk = (total + gridDim.x - 1) / gridDim.x;
    g_begin = static_cast<long long>(blockIdx.x) * chunk;
    g_end = min(total, g_begin + chunk);
    if (g_begin >= g_end) return;
  }

  int scan = P.boxes ? scan_of_tile(P, g_begin) : 0;
  int staged = -1;
  bool fits = false;
  int nlo = 0, cl_lo = 0, cl_hi = 0;
  // this thread's best argmax key over the CTA's tiles of the current scan;
  // the CTA reduces it once per scan, not once per tile
  unsigned long long run_key = 0ull;

  for (long long g = g_begin;; ++g) {
    if (g >= g_end) {
      if (!dyn) break;
      // the next chunk; every thread reads it after the barrier, and the
      // barrier before it keeps the previous chunk's values until all have
      __syncthreads();
      if (tid == 0) {
        const long long left = total - *reinterpret_cast<volatile int*>(P.work);
        const int c = static_cast<int>(max(2LL, left / (8LL * gridDim.x)));
        sInt[2] = atomicAdd(P.work, c);
        sInt[3] = c;
      }
      __syncthreads();
      g = sInt[2];
      if (g >= total) break;
      g_end = min(total, g + sInt[3]);
      if (P.boxes) scan = scan_of_tile(P, g);
    }
    long long t;
    if (P.boxes) {
      while (P.prefix[scan + 1] <= g) ++scan;
      t = g - P.prefix[scan];
    } else {
      scan = static_cast<int>(g / P.uni.tiles);
      t = g - static_cast<long long>(scan) * P.uni.tiles;
    }
    const LatBox L = P.boxes ? P.boxes[scan] : P.uni;

    if (scan != staged) {
      // ---- stage scan `scan`: descriptor, antennas, reachable sample window ----
      // literal DMAS lands a 16-bit window (ragged plans; uniform batches are
      // float32) in the (offset, fraction) table: order this thread's table
      // stores before the copy's async-proxy writes
      if constexpr (BF == BF_DMAS_LIT && RG)
        if (P.dtype != DT_F32) fence_proxy_async_smem();
      __syncthreads();  // every read of the previous window is complete
      if (tid == 0) {
        make_desc(P, scan, *sS);
        sInt[0] = INT_MAX;
        sInt[1] = INT_MIN;
      }
      __syncthreads();
      const int M = scan_M<RG>(P, sS), R = scan_R<RG>(P, sS);
      const float kscale = scan_kscale<RG>(P, sS);
      for (int j = tid; j < M; j += T) {
        const float* ga = sS->ant;
        sAnt[j] = make_float4(ga[3 * j + 0], ga[3 * j + 1], ga[3 * j + 2], 0.f);
      }
      if (BF == BF_DMAS_LIT)  // zero the padded antenna rows of this scan
        for (int j = tid; j < (rows - R) * P.span; j += T) sTr[R * P.span + j] = 0.f;
      __syncthreads();
      float bmin[3], bmax[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float p0 = fmaf(static_cast<float>(L.lo[a]), scan_pit<RG>(P, sS, a),
                              scan_org<RG>(P, sS, a));
        const float p1 = fmaf(static_cast<float>(L.lo[a] + L.step[a] * (L.cnt[a] - 1)),
                              scan_pit<RG>(P, sS, a), scan_org<RG>(P, sS, a));
        bmin[a] = fminf(p0, p1);
        bmax[a] = fmaxf(p0, p1);
      }
      // nearest and farthest distance from each antenna to the lattice's box
      for (int i = tid; i < M; i += T) {
        float dn2 = 0.f, df2 = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float av = a == 0 ? sAnt[i].x : (a == 1 ? sAnt[i].y : sAnt[i].z);
          const float dn = av - fminf(fmaxf(av, bmin[a]), bmax[a]);
          const float df = fmaxf(fabsf(av - bmin[a]), fabsf(av - bmax[a]));
          dn2 = fmaf(dn, dn, dn2);
          df2 = fmaf(df, df, df2);
        }
        if (MS) {
          sD[i] = sqrtf(dn2);  // scratch until the tile computation starts
          sD[M + i] = sqrtf(df2);
        } else {
          const float umin = fminf(fmaxf(sqrtf(dn2) * kscale - P.h, -1e8f), 1e8f);
          const float umax = fminf(fmaxf(sqrtf(df2) * kscale - P.h, -1e8f), 1e8f);
          atomicMin(&sInt[0], static_cast<int>(floorf(umin)) - 2);
          atomicMax(&sInt[1], static_cast<int>(floorf(umax)) + P.wpad + 3);
        }
      }
      if (MS) {
        __syncthreads();
        const float half_k = 0.5f * kscale;
        for (int r = tid; r < R; r += T) {
          const int2 c = sCh[r];
          const float umin = fminf(fmaxf((sD[c.x] + sD[c.y]) * half_k - P.h, -1e8f), 1e8f);
          const float umax =
              fminf(fmaxf((sD[M + c.x] + sD[M + c.y]) * half_k - P.h, -1e8f), 1e8f);
          atomicMin(&sInt[0], static_cast<int>(floorf(umin)) - 2);
          atomicMax(&sInt[1], static_cast<int>(floorf(umax)) + P.wpad + 3);
        }
      }
      __syncthreads();
      // TMA needs a 16-byte aligned sample coordinate (4 or 8 samples)
      nlo = sInt[0] & (P.dtype == DT_F32 ? ~3 : ~7);
      fits = (static_cast<long long>(sInt[1]) - nlo) <= P.span;
      cl_lo = nlo;
      // a thread reads samples n0 .. n0 + (window chunk) of the staged row
      cl_hi = nlo + P.span - 1 - ((BF == BF_DMAS_LIT) ? P.wpad : V);
      if (fits) {
        const int tma_index = sS->tma;
        if (tma_ok && tma_index >= 0) {
          if (tid == 0) {
            const CUtensorMap* map = P.tmaps ? P.tmaps + tma_index : &tmap;
            const int z = P.tmaps ? 0 : tma_index;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(
                bar, static_cast<uint32_t>(R) * P.span * static_cast<uint32_t>(dtype_bytes(P.dtype)));
            tma_load_3d(tma_dst, map, nlo - sS->n_begin, 0, z, bar);
          }
          uint32_t ok = 0;
          for (long it = 0; it < kWaitProbes && !ok; ++it) ok = mbar_try_wait(bar, phase);
          if (__syncthreads_or(!ok)) {
            // the copy did not land in time: record it, give the copy a last
            // bounded chance to finish (it writes this CTA's shared memory),
            // then leave without touching the outputs. The launch's results
            // are invalid from here on, so a counter-driven launch hands out
            // no more tiles (every later grab lands beyond the last tile).
            if (tid == 0) {
              atomicExch(P.status, UWB_ERR_TIMEOUT);
              if (dyn) atomicExch(P.work, INT_MAX / 2);
            }
            for (long it = 0; it < kWaitProbes && !ok; ++it) ok = mbar_try_wait(bar, phase);
            __syncthreads();
            return;
          }
          phase ^= 1u;
          if (P.dtype != DT_F32) {  // widen the 16-bit window
            const int total_s = R * P.span;
            const bool f16 = P.dtype == DT_F16;
            auto widen = [&](int j) {
              const unsigned short b = sRaw[j];
              return f16 ? __half2float(__ushort_as_half(b))
                         : __bfloat162float(__ushort_as_bfloat16(b));
            };
            if (BF == BF_DMAS_LIT && V <= 64) {  // the raw window sits in the delay table
              for (int j = tid; j < total_s; j += T) sTr[j] = widen(j);
            } else {
              // in place: the raw window starts at byte >= 2 * total_s of the
              // float window's area, so widening the elements [a, (total_s +
              // a) / 2 - 1) writes below every raw element from a on. Stages
              // of that size halve what remains; the last T or fewer elements
              // are read before any of them is written.
              int a = 0;
              while (total_s - a > T) {
                const int e = (total_s + a) / 2 - 1;
                for (int j = a + tid; j < e; j += T) sTr[j] = widen(j);
                __syncthreads();
                a = e;
              }
              const int j = a + tid;
              const float v = j < total_s ? widen(j) : 0.f;
              __syncthreads();
              if (j < total_s) sTr[j] = v;
            }
            __syncthreads();
          }
        } else {
          const ScanDesc S = *sS;
          const int total_s = R * P.span;
          for (int j = tid; j < total_s; j += T) {
            const int i = j / P.span;
            sTr[j] = sample_at(S, P.dtype, i, nlo + (j - i * P.span));
          }
          __syncthreads();
        }
      }
      staged = scan;
    }

    // ---- one tile of the lattice: linear or shaped ----
    int tix = 0, tiy = 0, tiz = 0;
    if (!linear) {
      const int ntx = (L.cnt[0] + P.tdim[0] - 1) / P.tdim[0];
      const int nty = (L.cnt[1] + P.tdim[1] - 1) / P.tdim[1];
      tix = static_cast<int>(t % ntx);
      tiy = static_cast<int>((t / ntx) % nty);
      tiz = static_cast<int>(t / (static_cast<long long>(ntx) * nty));
    }
    const int cxy = L.cnt[0] * L.cnt[1];
    int kx[PP], ky[PP], kz[PP];
    bool valid[PP];
    long long lin[PP];
    float px[PP], py[PP], pz[PP], energy[PP];
#pragma unroll
    for (int q = 0; q < PP; ++q) {
      if (linear) {
        // point t * (T * PP) + tid + q * T of the box
        const int idx = static_cast<int>(t) * (T * PP) + tid + q * T;
        if (P.strip > 1 && L.cnt[2] == 1) {
          // 2-D boxes with steep delays: strips of S rows numbered column by
          // column, so that a warp's 32 points form a block of 32 / S columns
          // by S rows whose delays span fewer than 32 samples (no two lanes
          // read words 32 apart: no shared-memory bank conflicts)
          const int S = P.strip;
          kz[q] = 0;
          valid[q] = idx < cxy;
          if (valid[q]) {
            const int sc = S * L.cnt[0];
            const int j = idx / sc;
            const int r = idx - j * sc;
            const int h = min(S, L.cnt[1] - S * j);
            kx[q] = r / h;
            ky[q] = S * j + (r - kx[q] * h);
          } else {
            kx[q] = ky[q] = 0;
          }
        } else {
          // x fastest
          kz[q] = idx / cxy;
          const int r = idx - kz[q] * cxy;
          ky[q] = r / L.cnt[0];
          kx[q] = r - ky[q] * L.cnt[0];
          valid[q] = kz[q] < L.cnt[2];
        }
      } else {
        kx[q] = tix * P.tdim[0] + lx[q];
        ky[q] = tiy * P.tdim[1] + ly[q];
        kz[q] = tiz * P.tdim[2] + lz[q];
        valid[q] = kx[q] < L.cnt[0] && ky[q] < L.cnt[1] && kz[q] < L.cnt[2];
      }
      const int gx = L.lo[0] + L.step[0] * kx[q];
      const int gy = L.lo[1] + L.step[1] * ky[q];
      const int gz = L.lo[2] + L.step[2] * kz[q];
      lin[q] = gx + static_cast<long long>(scan_gn<RG>(P, sS, 0)) *
                        (gy + static_cast<long long>(scan_gn<RG>(P, sS, 1)) * gz);
      px[q] = fmaf(static_cast<float>(gx), scan_pit<RG>(P, sS, 0), scan_org<RG>(P, sS, 0));
      py[q] = fmaf(static_cast<float>(gy), scan_pit<RG>(P, sS, 1), scan_org<RG>(P, sS, 1));
      pz[q] = fmaf(static_cast<float>(gz), scan_pit<RG>(P, sS, 2), scan_org<RG>(P, sS, 2));
      energy[q] = 0.f;
    }
    if constexpr (PP == 2) {
      // both points together (an invalid one is evaluated at its in-range
      // clamped samples and discarded)
      if (valid[0] || valid[1]) {
        if (fits) {
          const float2 e = energy_sum_pair<BF, V, RG, MS>(
              P, sS, sTr, sAnt, sCh, sD, nlo, cl_lo, cl_hi, make_float2(px[0], px[1]),
              make_float2(py[0], py[1]), make_float2(pz[0], pz[1]));
          energy[0] = e.x;
          energy[1] = e.y;
        } else {
#pragma unroll
          for (int q = 0; q < PP; ++q)
            if (valid[q])
              energy[q] = energy_sum_global<BF, V, MS>(P, sS, sAnt, sCh, sD, px[q], py[q], pz[q]);
        }
      }
    } else if (valid[0]) {
      if constexpr (BF == BF_DMAS_LIT) {
        if constexpr (V > 64) {
          energy[0] = fits ? energy_literal_blocks<V / 32, true, RG>(P, sS, sTr, sAnt, nlo, cl_lo,
                                                                     cl_hi, px[0], py[0], pz[0])
                           : energy_literal_blocks_global<V / 32, RG>(P, sS, sAnt, px[0], py[0],
                                                                      pz[0]);
        } else if constexpr (V <= 16) {
          energy[0] = fits ? energy_literal4<V, true, RG>(P, sS, sTr, sAnt, sNF, nlo, cl_lo, cl_hi,
                                                          px[0], py[0], pz[0])
                           : energy_literal_global<V>(P, sS, sAnt, sNF, px[0], py[0], pz[0]);
        } else if constexpr (RG) {
          // ragged plans size the block for their largest scan: each scan takes
          // the smallest pair-sample block that holds its own antennas, so a
          // small scan forms no products with zero rows beyond that block
          const int Ms = scan_M<RG>(P, sS);
          if (!fits)
            energy[0] = energy_literal_global<V>(P, sS, sAnt, sNF, px[0], py[0], pz[0]);
          else if (Ms <= 16)
            energy[0] = energy_literal<16, true, RG>(P, sS, sTr, sAnt, sNF, nlo, cl_lo, cl_hi,
                                                     px[0], py[0], pz[0]);
          else if (V > 32 && Ms <= 32)
            energy[0] = energy_literal<32, true, RG>(P, sS, sTr, sAnt, sNF, nlo, cl_lo, cl_hi,
                                                     px[0], py[0], pz[0]);
          else
            energy[0] = energy_literal<V, true, RG>(P, sS, sTr, sAnt, sNF, nlo, cl_lo, cl_hi,
                                                    px[0], py[0], pz[0]);
        } else {
          energy[0] = fits ? energy_literal<V, true, RG>(P, sS, sTr, sAnt, sNF, nlo, cl_lo, cl_hi,
                                                         px[0], py[0], pz[0])
                           : energy_literal_global<V>(P, sS, sAnt, sNF, px[0], py[0], pz[0]);
        }
      } else {
        energy[0] = fits ? energy_sum<BF, V, true, MS, RG>(P, sS, sTr, sAnt, sCh, sD, nlo, cl_lo,
                                                           cl_hi, px[0], py[0], pz[0])
                         : energy_sum_global<BF, V, MS>(P, sS, sAnt, sCh, sD, px[0], py[0], pz[0]);
      }
    }
    const long long img_off = RG ? sS->img_off : static_cast<long long>(scan) * P.gP;
    const long long cmp_off = RG ? sS->cmp_off : static_cast<long long>(scan) * P.compact_stride;
#pragma unroll
    for (int q = 0; q < PP; ++q) {
      if (!valid[q]) continue;
      if (P.image) {
        const long long gp = static_cast<long long>(scan_gn<RG>(P, sS, 0)) *
                             scan_gn<RG>(P, sS, 1) * scan_gn<RG>(P, sS, 2);
        P.image[img_off + check_run64(P.status, lin[q], gp)] = energy[q];
      }
      if (P.compact)
        P.compact[cmp_off +
                  check_run64(P.status,
                              kx[q] + static_cast<long long>(L.cnt[0]) *
                                          (ky[q] + static_cast<long long>(L.cnt[1]) * kz[q]),
                              static_cast<long long>(L.cnt[0]) * L.cnt[1] * L.cnt[2])] =
            energy[q];
    }
    if (P.keys) {
      // larger energy wins; equal energies -> lower linear index wins
#pragma unroll
      for (int q = 0; q < PP; ++q) {
        const unsigned long long key =
            valid[q] ? (static_cast<unsigned long long>(__float_as_uint(energy[q])) << 32) |
                           (0xFFFFFFFFull - static_cast<unsigned long long>(lin[q]))
                     : 0ull;
        run_key = key > run_key ? key : run_key;
      }
      // a range or chunk holds consecutive tiles: reduce when its last tile
      // of this scan is done (uniform across the CTA)
      const bool scan_ends =
          g + 1 == g_end || (P.boxes ? P.prefix[scan + 1] <= g + 1
                                     : (g + 1) % P.uni.tiles == 0);
      if (scan_ends) {
        unsigned long long k = run_key;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const unsigned long long other = __shfl_xor_sync(0xFFFFFFFFu, k, o);
          k = other > k ? other : k;
        }
        if (lane == 0) sKey[warp] = k;
        __syncthreads();
        if (tid == 0) {
          unsigned long long best = 0;
          for (int w = 0; w < (T >> 5); ++w) best = sKey[w] > best ? sKey[w] : best;
          if (best) atomicMax(P.keys + scan, best);
        }
        __syncthreads();
        run_key = 0ull;
      }
    }
  }
}

// Instance selection: ragged batches (descriptors present) run the RG
// instance; multistatic batches the MS one.
template <int BF, int V, bool MS>
cudaError_t launch_variant(const ImgParams& p, const CUtensorMap* tmap, int ctas, int threads,
                           size_t smem, cudaStream_t st) {
  if constexpr (!MS) {
    if (p.descs) {
      k_image<BF, V, false, true><<<ctas, threads, smem, st>>>(*tmap, p);
      return cudaGetLastError();
    }
  }
  k_image<BF, V, MS, false><<<ctas, threads, smem, st>>>(*tmap, p);
  return cudaGetLastError();
}

// The instance's dynamic shared-memory limit is raised to the device's
// opt-in maximum (it is only a ceiling), so that launches of any smaller size
// stay valid whichever size was queried last.
template <int BF, int V, bool MS, bool RG>
int occupancy_instance(int threads, size_t smem) {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  if (smem > static_cast<size_t>(optin)) return 0;
  if (cudaFuncSetAttribute(k_image<BF, V, MS, RG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin) != cudaSuccess)
    return 0;
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_image<BF, V, MS, RG>, threads,
                                                    smem) != cudaSuccess)
    return 0;
  return blocks;
}

// Resident CTAs of the instance a launch will use: the ragged one (per-scan
// descriptors, monostatic only) or the uniform one.
template <int BF, int V, bool MS>
int occupancy_variant(bool rg, int threads, size_t smem) {
  if constexpr (!MS) {
    if (rg) return occupancy_instance<BF, V, false, true>(threads, smem);
  }
  return occupancy_instance<BF, V, MS, false>(threads, smem);
}

}  // namespace uwb
