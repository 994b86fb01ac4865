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
//  * one thread per focal point; the delay is computed in registers, the
//    W+1 samples of the window are read from shared memory and interpolated;
//  * fused epilogue: image store, compact-profile store, and a block-reduced
//    64-bit (energy, -index) key folded into the scan's argmax with atomicMax.
// Scans whose window does not fit the staged span fall back to bounds-checked
// global loads (same arithmetic).
#pragma once

#include <climits>

#include "ptx.cuh"
#include "uwb_internal.cuh"

namespace uwb {

// Bounded waits: a staging wait gives up after this many try_wait probes.
constexpr long kWaitProbes = 1L << 24;

template <int BF, int V>
struct KernelShape {
  static constexpr int threads = (BF == BF_DMAS_LIT) ? 128 : 256;
  // literal DMAS: 4 resident CTAs (<= 128 registers) up to 32 antennas
  static constexpr int min_blocks = (BF == BF_DMAS_LIT) ? (V <= 32 ? 4 : 2) : (BF == BF_DAS ? (V <= 20 ? 4 : 3) : (V <= 20 ? 3 : 2));
};

// -------------------------------------------------------------- DAS / DMAS-identity
// Rows are the M antennas (monostatic: delay 2|r - a_i| fs / v) or, with MS,
// the R channels (transmitter, receiver) of a multistatic recording (Eq. 2:
// delay (|r - a_tx| + |r - a_rx|) fs / v); for MS each thread first puts its
// focal point's distance to every antenna in sD[antenna][thread].
template <int BF, int WT, bool STAGED, bool MS>
__device__ __forceinline__ float energy_sum(const ImgParams& P, const float* __restrict__ sTr,
                                            const float4* __restrict__ sAnt,
                                            const int2* __restrict__ sCh, float* __restrict__ sD,
                                            const float* __restrict__ gTr, int nlo, int cl_lo,
                                            int cl_hi, float px, float py, float pz) {
  float energy = 0.f;
  const int R = P.R;
  const int T = blockDim.x, tid = threadIdx.x;
  if (MS) {
    for (int i = 0; i < P.M; ++i) {
      const float4 a = sAnt[i];
      const float dx = px - a.x, dy = py - a.y, dz = pz - a.z;
      sD[i * T + tid] = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    }
  }
  const float half_k = 0.5f * P.kscale;
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
        const float d = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        t = fmaf(d, P.kscale, -hoff);
      }
      const float fl = floorf(t);
      const float f = t - fl;
      int n0 = static_cast<int>(fl);
      float y[WT + 1];
      if (STAGED) {
        n0 = min(max(n0, cl_lo), cl_hi);
        const float* row = sTr + i * P.span + (n0 - nlo);
#pragma unroll
        for (int k = 0; k <= WT; ++k) y[k] = row[k];
      } else {
        const float* row = gTr + static_cast<size_t>(i) * P.pitch;
#pragma unroll
        for (int k = 0; k <= WT; ++k) {
          const int n = n0 + k - P.n_begin;
          y[k] = (n >= 0 && n < P.N) ? __ldg(row + n) : 0.f;
        }
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

template <bool STAGED>
__device__ __forceinline__ LitRaw lit_load(const ImgParams& P, const float* __restrict__ sTr,
                                           const float2* __restrict__ sNF,
                                           const float* __restrict__ gTr, int i, int T, int tid,
                                           int k0) {
  const float2 nf = sNF[i * T + tid];
  const int off = __float_as_int(nf.x) + k0;
  LitRaw r;
  r.f = nf.y;
  if (STAGED) {
    const float* row = sTr + i * P.span + off;
    r.y0 = row[0];
    r.y1 = row[1];
    r.y2 = row[2];
  } else if (i < P.M) {
    const float* row = gTr + static_cast<size_t>(i) * P.pitch;
    const int o = off - P.n_begin;
    r.y0 = (o >= 0 && o < P.N) ? __ldg(row + o) : 0.f;
    r.y1 = (o + 1 >= 0 && o + 1 < P.N) ? __ldg(row + o + 1) : 0.f;
    r.y2 = (o + 2 >= 0 && o + 2 < P.N) ? __ldg(row + o + 2) : 0.f;
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

// sTr holds MMAX rows; rows M..MMAX-1 are zero (written at kernel start).
template <int MMAX, bool STAGED>
__device__ __forceinline__ float energy_literal(const ImgParams& P, const float* __restrict__ sTr,
                                                const float4* __restrict__ sAnt,
                                                float2* __restrict__ sNF,
                                                const float* __restrict__ gTr, int nlo,
                                                int cl_lo, int cl_hi, float px, float py,
                                                float pz) {
  const int T = blockDim.x, tid = threadIdx.x;
  const int M = P.M;
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
      const float d = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
      const float t = fmaf(d, P.kscale, -hf);
      const float fl = floorf(t);
      f = t - fl;
      n0 = static_cast<int>(fl);
      if (STAGED) n0 = min(max(n0, cl_lo), cl_hi) - nlo;
    }
    sNF[i * T + tid] = make_float2(__int_as_float(n0), f);
  }
  float energy = 0.f;
  for (int k0 = 0; k0 < P.W; k0 += 2) {
    float2 x[MMAX];
    float2 acc[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) acc[a] = make_float2(0.f, 0.f);
    LitRaw next = lit_load<STAGED>(P, sTr, sNF, gTr, 0, T, tid, k0);
#pragma unroll
    for (int j = 0; j < MMAX; ++j) {
      const LitRaw cur = next;
      if (j + 1 < MMAX) next = lit_load<STAGED>(P, sTr, sNF, gTr, j + 1, T, tid, k0);
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

// ------------------------------------------------------------------ the kernel
// V = window chunk WT (DAS, DMAS identity) or antenna register block MMAX
// (literal DMAS); MS = multistatic rows. Dynamic shared memory (see
// image_smem_bytes): [rows][span] traces | [M] antennas (float4) | (MS) [R]
// channels | (literal) [V][T] delays | (MS) [M][T] distances | mbarrier and
// reduction slots.
template <int BF, int V, bool MS>
__global__ void __launch_bounds__(KernelShape<BF, V>::threads, KernelShape<BF, V>::min_blocks)
    k_image(const __grid_constant__ CUtensorMap tmap, const ImgParams P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int T = blockDim.x, tid = threadIdx.x;
  const int M = P.M;
  const int R = P.R;  // trace rows per scan: M antennas, or R channels
  // literal DMAS keeps V (>= M) trace rows; rows M..V-1 stay zero
  const int rows = (BF == BF_DMAS_LIT) ? V : R;
  float* sTr = reinterpret_cast<float*>(smem_raw);
  // antennas as (x, y, z, 0): one broadcast 16-byte load per antenna
  float4* sAnt = reinterpret_cast<float4*>(sTr + static_cast<size_t>(rows) * P.span);
  int2* sCh = reinterpret_cast<int2*>(sAnt + M);
  float2* sNF = reinterpret_cast<float2*>(sCh + (MS ? R : 0));
  const size_t nf_words = (BF == BF_DMAS_LIT) ? static_cast<size_t>(V) * T * 2 : 0;
  float* sD = reinterpret_cast<float*>(sNF) + nf_words;
  const size_t d_words = MS ? static_cast<size_t>(M) * T : 0;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sD + d_words);
  unsigned long long* sKey = reinterpret_cast<unsigned long long*>(bar + 1);  // [32]
  int* sInt = reinterpret_cast<int*>(sKey + 32);                              // [4]

  // thread -> point of the tile (warp sub-blocks of wdim points)
  const int lane = tid & 31, warp = tid >> 5;
  const int nbx = P.tdim[0] / P.wdim[0], nby = P.tdim[1] / P.wdim[1];
  const int lx = (warp % nbx) * P.wdim[0] + lane % P.wdim[0];
  const int ly = ((warp / nbx) % nby) * P.wdim[1] + (lane / P.wdim[0]) % P.wdim[1];
  const int lz = (warp / (nbx * nby)) * P.wdim[2] + lane / (P.wdim[0] * P.wdim[1]);

  const bool tma_ok = P.use_tma && ((smem_u32(sTr) & 127u) == 0);
  if (tid == 0) mbar_init(bar, 1);
  if (BF == BF_DMAS_LIT)
    for (int j = tid; j < (rows - M) * P.span; j += T) sTr[M * P.span + j] = 0.f;
  if (MS) {
    // channel table (shared by every scan); indices outside the array are
    // recorded as an argument error and clamped so that no access leaves it
    for (int r = tid; r < R; r += T) {
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
  const long long chunk = (total + gridDim.x - 1) / gridDim.x;
  const long long g_begin = static_cast<long long>(blockIdx.x) * chunk;
  const long long g_end = min(total, g_begin + chunk);
  if (g_begin >= g_end) return;

  int scan = 0;
  if (P.boxes) {  // largest scan with prefix[scan] <= g_begin
    int lo = 0, hi = P.B;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (P.prefix[mid] <= g_begin) lo = mid; else hi = mid;
    }
    scan = lo;
  }
  int staged = -1;
  bool fits = false;
  int nlo = 0, cl_lo = 0, cl_hi = 0;
  const float* gTr = nullptr;

  for (long long g = g_begin; g < g_end; ++g) {
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
      // ---- stage scan `scan`: antennas, reachable sample window ----
      __syncthreads();  // every read of the previous window is complete
      const float* ga = P.ant + static_cast<long long>(scan) * P.ant_stride;
      for (int j = tid; j < M; j += T)
        sAnt[j] = make_float4(ga[3 * j + 0], ga[3 * j + 1], ga[3 * j + 2], 0.f);
      if (tid == 0) {
        sInt[0] = INT_MAX;
        sInt[1] = INT_MIN;
      }
      __syncthreads();
      float bmin[3], bmax[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float p0 = fmaf(static_cast<float>(L.lo[a]), P.pit[a], P.org[a]);
        const float p1 =
            fmaf(static_cast<float>(L.lo[a] + L.step[a] * (L.cnt[a] - 1)), P.pit[a], P.org[a]);
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
          const float umin = fminf(fmaxf(sqrtf(dn2) * P.kscale - P.h, -1e8f), 1e8f);
          const float umax = fminf(fmaxf(sqrtf(df2) * P.kscale - P.h, -1e8f), 1e8f);
          atomicMin(&sInt[0], static_cast<int>(floorf(umin)) - 2);
          atomicMax(&sInt[1], static_cast<int>(floorf(umax)) + P.wpad + 3);
        }
      }
      if (MS) {
        __syncthreads();
        const float half_k = 0.5f * P.kscale;
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
      nlo = sInt[0] & ~3;  // TMA needs a 16-byte aligned sample coordinate
      fits = (static_cast<long long>(sInt[1]) - nlo) <= P.span;
      cl_lo = nlo;
      // a thread reads samples n0 .. n0 + (window chunk) of the staged row
      cl_hi = nlo + P.span - 1 - ((BF == BF_DMAS_LIT) ? P.wpad : V);
      gTr = P.traces + static_cast<long long>(scan) * P.trace_stride;
      if (fits) {
        if (tma_ok) {
          if (tid == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, static_cast<uint32_t>(R) * P.span * 4u);
            tma_load_3d(sTr, &tmap, nlo - P.n_begin, 0, scan, bar);
          }
          uint32_t ok = 0;
          for (long it = 0; it < kWaitProbes && !ok; ++it) ok = mbar_try_wait(bar, phase);
          if (__syncthreads_or(!ok)) {
            // the copy did not land in time: record it, give the copy a last
            // bounded chance to finish (it writes this CTA's shared memory),
            // then leave without touching the outputs.
            if (tid == 0) atomicExch(P.status, UWB_ERR_TIMEOUT);
            for (long it = 0; it < kWaitProbes && !ok; ++it) ok = mbar_try_wait(bar, phase);
            __syncthreads();
            return;
          }
          phase ^= 1u;
        } else {
          const int total_s = R * P.span;
          for (int j = tid; j < total_s; j += T) {
            const int i = j / P.span;
            const int n = nlo + (j - i * P.span) - P.n_begin;
            sTr[j] = (n >= 0 && n < P.N) ? gTr[static_cast<size_t>(i) * P.pitch + n] : 0.f;
          }
          __syncthreads();
        }
      }
      staged = scan;
    }

    // ---- one tile of the lattice ----
    const int ntx = (L.cnt[0] + P.tdim[0] - 1) / P.tdim[0];
    const int nty = (L.cnt[1] + P.tdim[1] - 1) / P.tdim[1];
    const int tix = static_cast<int>(t % ntx);
    const int tiy = static_cast<int>((t / ntx) % nty);
    const int tiz = static_cast<int>(t / (static_cast<long long>(ntx) * nty));
    const int kx = tix * P.tdim[0] + lx, ky = tiy * P.tdim[1] + ly, kz = tiz * P.tdim[2] + lz;
    const bool valid = kx < L.cnt[0] && ky < L.cnt[1] && kz < L.cnt[2];
    const int gx = L.lo[0] + L.step[0] * kx;
    const int gy = L.lo[1] + L.step[1] * ky;
    const int gz = L.lo[2] + L.step[2] * kz;
    const long long lin =
        gx + static_cast<long long>(P.gn[0]) * (gy + static_cast<long long>(P.gn[1]) * gz);
    float energy = 0.f;
    if (valid) {
      const float px = fmaf(static_cast<float>(gx), P.pit[0], P.org[0]);
      const float py = fmaf(static_cast<float>(gy), P.pit[1], P.org[1]);
      const float pz = fmaf(static_cast<float>(gz), P.pit[2], P.org[2]);
      if constexpr (BF == BF_DMAS_LIT) {
        energy = fits ? energy_literal<V, true>(P, sTr, sAnt, sNF, gTr, nlo, cl_lo, cl_hi, px,
                                                py, pz)
                      : energy_literal<V, false>(P, sTr, sAnt, sNF, gTr, nlo, cl_lo, cl_hi,
                                                 px, py, pz);
      } else {
        energy = fits ? energy_sum<BF, V, true, MS>(P, sTr, sAnt, sCh, sD, gTr, nlo, cl_lo,
                                                    cl_hi, px, py, pz)
                      : energy_sum<BF, V, false, MS>(P, sTr, sAnt, sCh, sD, gTr, nlo, cl_lo,
                                                     cl_hi, px, py, pz);
      }
      if (P.image) P.image[static_cast<long long>(scan) * P.gP + lin] = energy;
      if (P.compact)
        P.compact[static_cast<long long>(scan) * P.compact_stride + kx +
                  static_cast<long long>(L.cnt[0]) * (ky + static_cast<long long>(L.cnt[1]) * kz)] =
            energy;
    }
    if (P.keys) {
      // larger energy wins; equal energies -> lower linear index wins
      unsigned long long key =
          valid ? (static_cast<unsigned long long>(__float_as_uint(energy)) << 32) |
                      (0xFFFFFFFFull - static_cast<unsigned long long>(lin))
                : 0ull;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xFFFFFFFFu, key, o);
        key = other > key ? other : key;
      }
      if (lane == 0) sKey[warp] = key;
      __syncthreads();
      if (tid == 0) {
        unsigned long long best = 0;
        for (int w = 0; w < (T >> 5); ++w) best = sKey[w] > best ? sKey[w] : best;
        if (best) atomicMax(P.keys + scan, best);
      }
      __syncthreads();
    }
  }
}

template <int BF, int V, bool MS>
cudaError_t launch_variant(const ImgParams& p, const CUtensorMap* tmap, int ctas, int threads,
                           size_t smem, cudaStream_t st) {
  k_image<BF, V, MS><<<ctas, threads, smem, st>>>(*tmap, p);
  return cudaGetLastError();
}

template <int BF, int V, bool MS>
int occupancy_variant(int threads, size_t smem) {
  if (cudaFuncSetAttribute(k_image<BF, V, MS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess)
    return 0;
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_image<BF, V, MS>, threads,
                                                    smem) != cudaSuccess)
    return 0;
  return blocks;
}

}  // namespace uwb
