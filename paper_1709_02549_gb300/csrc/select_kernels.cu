// Device-resident segment search (Section III, "ROI Selection"): one warp (or,
// for large batches of small profiles, a quarter warp) per scan runs the
// whole coarse-to-fine loop on the decimated energy profile --
// quadrant/octant split, per-child mean and variance (compensated float32
// sums finished in float64), the Eq. 5 decision metric, sliding framing of
// the chosen child, and the Eq. 6-7 stopping rule -- then writes the final
// region as a lattice box for the full-resolution pass. No host round trip
// between steps.
//
// Readings where the paper is silent or inconsistent (the same ones the
// float64 reference implementation takes):
//  * energies are divided by the profile maximum before any metric (Eq. 5
//    adds a mean to a variance, which is only scale-free after normalising);
//  * sigma^2_{i-1} of Eq. 5 is the variance of the region being split (the
//    whole region at the first iteration); population variance; a child with
//    zero variance scores its mean; the Eq. 5 weight is clipped to [0, 1]
//    (UWB_METRIC_HYBRID) or used as printed (UWB_METRIC_HYBRID_UNCLIPPED);
//  * the two classes of Eq. 6-7 are the decimated energies of the regions of
//    consecutive iterations; the loop continues while B grows and W shrinks,
//    tested from the second iteration, and returns the last accepted region;
//  * children without a decimated point or with a side below min_segment are
//    not candidates; ties go to the lowest child index (bit 0 = high x half,
//    bit 1 = high y, bit 2 = high z).
#include "uwb_internal.cuh"

namespace uwb {
namespace {

// Decimated-lattice index range [klo, khi) per axis of the points inside a
// full-resolution box [lo, hi).
struct KBox {
  int klo[3], khi[3];
  long long n;
};

__device__ KBox lattice_in_box(const SelScan& P, const int lo[3], const int hi[3]) {
  KBox b;
  b.n = 1;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int s = P.step[a];
    const int dl = lo[a] - P.off[a], dh = hi[a] - P.off[a];
    int kl = dl <= 0 ? 0 : (dl + s - 1) / s;
    int kh = dh <= 0 ? 0 : (dh + s - 1) / s;
    kl = min(kl, P.cnt[a]);
    kh = min(kh, P.cnt[a]);
    if (kh < kl) kh = kl;
    b.klo[a] = kl;
    b.khi[a] = kh;
    b.n *= (kh - kl);
  }
  return b;
}

// Visits the decimated points j = start, start + stride, ... of a box (x
// fastest) without dividing per point: the index is decomposed once and then
// advanced by the stride with carries (stride <= 32).
template <class F>
__device__ __forceinline__ void for_box_points(const KBox& b, int start, int stride, F&& f) {
  const int n = static_cast<int>(b.n);
  if (start >= n) return;
  const int nx = b.khi[0] - b.klo[0], ny = b.khi[1] - b.klo[1];
  int kx = start % nx, ky = (start / nx) % ny, kz = start / (nx * ny);
  const int sx = stride % nx, sy = stride / nx;
  for (int j = start; j < n; j += stride) {
    f(b.klo[0] + kx, b.klo[1] + ky, b.klo[2] + kz);
    kx += sx;
    ky += sy;
    if (kx >= nx) {
      kx -= nx;
      ++ky;
    }
    while (ky >= ny) {
      ky -= ny;
      ++kz;
    }
  }
}

// Normalisation by 1 / m (m = the profile maximum) in two parts, so that the
// work per lattice point stays in float32 (float64 is this GPU's slow path,
// about two lanes per clock per SM): e = I * 2^k exactly (m 2^k in [0.5, 1),
// applied as two float32 power-of-two factors), sums of e and e^2 carried as
// compensated float32 pairs, and the finished sums scaled by r = 2^-k / m in
// float64. Energies below 2^-126 of the maximum underflow in e^2; they add
// less than 1e-37 of the sums.
struct Norm {
  float sa, sb;
  double r;
};

__device__ __forceinline__ Norm make_norm(float m) {
  int ex;
  frexpf(m, &ex);  // m = f 2^ex, f in [0.5, 1); ex in [-148, 128]
  const int k = -ex, k1 = k / 2, k2 = k - k1;
  Norm n;
  n.sa = __int_as_float((k1 + 127) << 23);
  n.sb = __int_as_float((k2 + 127) << 23);
  n.r = ldexp(1.0 / static_cast<double>(m), -k);
  return n;
}

// A float32 sum carried with its rounding error (hi + lo; Knuth's two-sum
// recovers each addition's error exactly): about 48 significant bits.
struct Acc2 {
  float hi, lo;
};

__device__ __forceinline__ float two_sum_err(float a, float b, float s) {
  const float bv = s - a;
  return (a - (s - bv)) + (b - bv);
}

__device__ __forceinline__ void acc_add(Acc2& a, float b) {
  const float s = a.hi + b;
  a.lo += two_sum_err(a.hi, b, s);
  a.hi = s;
}

// e^2 as the product and its exact error (a fused multiply-add)
__device__ __forceinline__ void acc_sq(Acc2& a, float e) {
  const float p = e * e;
  acc_add(a, p);
  a.lo += fmaf(e, e, -p);
}

// Symmetric in its operands (the two-sum error is exact either way), so the
// lanes of a butterfly reduction end with the same value.
__device__ __forceinline__ Acc2 acc_merge(const Acc2& a, const Acc2& b) {
  const float s = a.hi + b.hi;
  return Acc2{s, (a.lo + b.lo) + two_sum_err(a.hi, b.hi, s)};
}

__device__ __forceinline__ Acc2 acc_shfl_xor(const Acc2& a, int o) {
  return Acc2{__shfl_xor_sync(0xFFFFFFFFu, a.hi, o), __shfl_xor_sync(0xFFFFFFFFu, a.lo, o)};
}

__device__ __forceinline__ double acc_value(const Acc2& a) {
  return static_cast<double>(a.hi) + static_cast<double>(a.lo);
}

struct Stats {
  long long n;
  // of the normalised energies; scatter = sum of squared deviations,
  // var = scatter / n (population variance)
  double sum, mean, scatter, var;
};

// Lane-partial sums of e and e^2 (e = I 2^k, see Norm) over the decimated
// points j = start, start + stride, ... of a box (one pass).
__device__ __forceinline__ void lane_sums(const SelScan& P, const float* prof, const KBox& b,
                                          const Norm& nm, int start, int stride, Acc2& a1,
                                          Acc2& a2) {
  a1 = Acc2{0.f, 0.f};
  a2 = Acc2{0.f, 0.f};
  for_box_points(b, start, stride, [&](int kx, int ky, int kz) {
    const float e = (prof[kx + P.cnt[0] * (ky + P.cnt[1] * kz)] * nm.sa) * nm.sb;
    acc_add(a1, e);
    acc_sq(a2, e);
  });
}

// Statistics of the normalised energies I / m (m = the profile maximum)
// inside a box: count, sum, mean, scatter (sum of squared deviations, as
// sum e^2 - (sum e) mean; the energies are non-negative and bounded, and the
// sums carry about 48 significant bits, so even nearly flat segments keep
// ~14 digits) and variance, finished in float64: one pass, and one division
// (1 / n) per box. The SW lanes of the scan's sub-warp (sl = lane in it)
// share the points; every lane of the warp takes part in the shuffles.
template <int SW>
__device__ Stats box_stats(const SelScan& P, const float* prof, const Norm& nm, const KBox& b,
                           int sl) {
  Stats st;
  st.n = b.n;
  st.sum = st.mean = st.scatter = st.var = 0.0;
  // the division first: its float64 latency passes during the point sums
  const double rn = 1.0 / static_cast<double>(b.n > 0 ? b.n : 1);
  Acc2 a1, a2;
  lane_sums(P, prof, b, nm, sl, SW, a1, a2);
#pragma unroll
  for (int o = SW / 2; o > 0; o >>= 1) {
    a1 = acc_merge(a1, acc_shfl_xor(a1, o));
    a2 = acc_merge(a2, acc_shfl_xor(a2, o));
  }
  if (b.n == 0) return st;
  st.sum = acc_value(a1) * nm.r;
  st.mean = st.sum * rn;
  st.scatter = fmax(acc_value(a2) * nm.r * nm.r - st.sum * st.mean, 0.0);
  st.var = st.scatter * rn;
  return st;
}

// Batches of at least this many scans, with at most this many decimated
// points per scan, select with four scans per warp.
constexpr int kSelectPackedMinScans = 2048;
constexpr long long kSelectPackedMaxPoints = 4096;

__device__ __forceinline__ double rel_gap(double hi, double lo) {
  const double d = fmax(fabs(hi), fabs(lo));
  return d == 0.0 ? 0.0 : (hi - lo) / d;
}

__device__ double decision_metric(int metric, double mu, double var, double var_prev) {
  if (metric == UWB_METRIC_MEAN) return mu;
  if (metric == UWB_METRIC_VARIANCE) return var;
  if (var == 0.0) return mu;
  double a = (var - var_prev) / var;  // Eq. 5 weight
  if (metric == UWB_METRIC_HYBRID) a = fmin(fmax(a, 0.0), 1.0);
  return (1.0 - a) * mu + a * var;
}

// Child choice of one iteration (Eq. 5 over the 2^dim children of the region
// [Rlo, Rhi)), all children at once: lane group c = sl / G of the scan's
// sub-warp (G = SW / 2^dim lanes, sl = lane in the sub-warp, base = its first
// lane) sums child c's lattice points, the group's sums are reduced within
// the group, and every lane then runs the choice over the children in index
// order (first maximum wins; the runner-up is kept for the margin).
struct Choice {
  int best, nvalid;
  double best_m, second_m;
  int blo[3], bhi[3];
};

template <int SW>
__device__ Choice choose_child(const SelScan& Q, const float* vals, const Norm& nm,
                               const int Rlo[3], const int Rhi[3], int dim,
                               const uwb_rule& rule, double var_prev, int sl, int base) {
  const int nchild = 1 << dim;
  const int G = SW / nchild;
  const int c = sl / G, r = sl % G;
  int mid[3], clo[3], chi[3];
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    mid[a] = Rlo[a] + (Rhi[a] - Rlo[a]) / 2;
    if (a < dim) {
      const int bit = (c >> a) & 1;
      clo[a] = bit ? mid[a] : Rlo[a];
      chi[a] = bit ? Rhi[a] : mid[a];
      if (chi[a] - clo[a] < rule.min_segment) ok = false;
    } else {
      clo[a] = Rlo[a];
      chi[a] = Rhi[a];
    }
  }
  const KBox kb = lattice_in_box(Q, clo, chi);
  const double rn = 1.0 / static_cast<double>(kb.n > 0 ? kb.n : 1);  // before the sums
  // this group's partial sums over child c
  Acc2 a1{0.f, 0.f}, a2{0.f, 0.f};
  if (ok) lane_sums(Q, vals, kb, nm, r, G, a1, a2);
  for (int o = G >> 1; o > 0; o >>= 1) {
    a1 = acc_merge(a1, acc_shfl_xor(a1, o));
    a2 = acc_merge(a2, acc_shfl_xor(a2, o));
  }
  double m = 0.0;
  const bool valid = ok && kb.n > 0;
  if (valid) {
    const double sum = acc_value(a1) * nm.r;
    const double mean = sum * rn;
    const double scatter = fmax(acc_value(a2) * nm.r * nm.r - sum * mean, 0.0);
    m = decision_metric(rule.metric, mean, scatter * rn, var_prev);
  }
  Choice ch;
  ch.best = -1;
  ch.nvalid = 0;
  ch.best_m = ch.second_m = 0.0;
  for (int a = 0; a < 3; ++a) ch.blo[a] = ch.bhi[a] = 0;
  // unrolled over the most children (8), so that every shuffle is issued
  // ahead of the compare chain
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) {
    if (cc >= nchild) break;
    const double mc = __shfl_sync(0xFFFFFFFFu, m, base + cc * G);
    const int vc = __shfl_sync(0xFFFFFFFFu, valid ? 1 : 0, base + cc * G);
    if (!vc) continue;
    if (ch.nvalid == 0 || mc > ch.best_m) {
      if (ch.nvalid > 0) ch.second_m = ch.best_m;
      ch.best_m = mc;
      ch.best = cc;
    } else if (ch.nvalid == 1 || mc > ch.second_m) {
      ch.second_m = mc;
    }
    ++ch.nvalid;
  }
  if (ch.best >= 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a < dim) {
        const int bit = (ch.best >> a) & 1;
        ch.blo[a] = bit ? mid[a] : Rlo[a];
        ch.bhi[a] = bit ? Rhi[a] : mid[a];
      } else {
        ch.blo[a] = Rlo[a];
        ch.bhi[a] = Rhi[a];
      }
    }
  }
  return ch;
}

// One scan per sub-warp of SW lanes: SW = 32, a warp per scan; SW = 8, four
// scans per warp. A scan's float32 point sums spread over its sub-warp's
// lanes, while the float64 finishing (one division per box, Eq. 5, Eq. 6-7)
// of all of a warp's scans runs as one instruction stream: float64 is this
// GPU's slow pipe, and with one scan per warp every lane repeats its scan's
// scalar finishing. A sub-warp without a scan to run (past the batch,
// skipped, no target, or stopped earlier than the others) keeps taking part
// in the shuffles on empty boxes, with its results and stores switched off.
template <int SW>
__global__ void __launch_bounds__(256) k_select(const SelParams P) {
  const int lane = threadIdx.x & 31, sl = lane & (SW - 1), base = lane - sl;
  const int s = static_cast<int>((static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) / SW);
  const bool in = s < P.B && !(P.skip && P.skip[s]);
  // this scan's lattice and grid (an empty lattice for a sub-warp without one)
  SelScan Q;
  if (!in) {
    Q.prof_off = 0;
    for (int a = 0; a < 3; ++a) {
      Q.gn[a] = 1;
      Q.off[a] = 0;
      Q.step[a] = 1;
      Q.cnt[a] = 0;
    }
    Q.D = 1;
    Q.max_iters = 0;
  } else if (P.scans) {
    Q = P.scans[s];
  } else {
    Q.prof_off = static_cast<long long>(s) * P.prof_stride;
    for (int a = 0; a < 3; ++a) {
      Q.gn[a] = P.gn[a];
      Q.off[a] = P.off[a];
      Q.step[a] = P.step[a];
      Q.cnt[a] = P.cnt[a];
    }
    Q.D = P.D;
    Q.max_iters = P.max_iters;
  }
  const float* prof = P.profile + Q.prof_off;
  uwb_result* R = P.out + (in ? s : 0);
  LatBox* box = P.boxes + (in ? s : 0);

  // clear the result record
  if (in) {
    int* w = reinterpret_cast<int*>(R);
    for (int j = sl; j < static_cast<int>(sizeof(uwb_result) / 4); j += SW) w[j] = 0;
  }
  __syncwarp();
  const long long Pd = static_cast<long long>(Q.cnt[0]) * Q.cnt[1] * Q.cnt[2];
  float fmx = 0.f;
  int bad = 0;
  for (long long j = sl; j < Pd; j += SW) {
    const float v = prof[j];
    bad |= !isfinite(v);
    fmx = fmaxf(fmx, v);
  }
#pragma unroll
  for (int o = SW / 2; o > 0; o >>= 1) {
    bad |= __shfl_xor_sync(0xFFFFFFFFu, bad, o);
    fmx = fmaxf(fmx, __shfl_xor_sync(0xFFFFFFFFu, fmx, o));
  }

  if (in && sl == 0) {
    R->decim = Q.D;
    for (int a = 0; a < 3; ++a) {
      R->offset[a] = Q.off[a];
      R->dcount[a] = Q.cnt[a];
      R->loc_idx[a] = -1;
    }
    R->profile_max = fmx;
    if (bad || fmx == 0.f) {
      R->status = bad ? UWB_ERR_NONFINITE : UWB_OK;
      R->stop_reason = bad ? UWB_STOP_NONE : UWB_STOP_NO_TARGET;
      for (int a = 0; a < 3; ++a) {
        box->lo[a] = 0;
        box->step[a] = 1;
        box->cnt[a] = 0;
      }
      box->tiles = 0;
    }
  }
  const bool live = in && !bad && fmx != 0.f;
  if (!__any_sync(0xFFFFFFFFu, live)) return;
  const Norm nm = make_norm(live ? fmx : 1.f);
  const int dim = P.dim;
  const uwb_rule& rule = P.rule;

  int Rlo[3] = {0, 0, 0}, Rhi[3] = {Q.gn[0], Q.gn[1], Q.gn[2]};
  Stats sa = box_stats<SW>(Q, prof, nm, lattice_in_box(Q, Rlo, Rhi), sl);
  double var_prev = sa.var;
  double B_prev = 0.0, W_prev = 0.0;
  int iters = 0, n_logged = 0, stop = UWB_STOP_NONE;
  bool run = live && Q.max_iters >= 1;

  for (int i = 1; __any_sync(0xFFFFFFFFu, run); ++i) {
    const int li = i - 1;
    const Choice ch = choose_child<SW>(Q, prof, nm, Rlo, Rhi, dim, rule, var_prev, sl, base);
    const int best = ch.best, nvalid = ch.nvalid;
    const double best_m = ch.best_m, second_m = ch.second_m;
    if (run && nvalid == 0) {
      stop = UWB_STOP_MINSIZE;
      iters = i - 1;
      run = false;
    }
    // sliding framing of the chosen child
    int Nlo[3], Nhi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a < dim) {
        const int side = ch.bhi[a] - ch.blo[a];
        const int grow = (side * rule.frame_num + rule.frame_den - 1) / rule.frame_den;
        Nlo[a] = max(ch.blo[a] - grow, 0);
        Nhi[a] = min(ch.bhi[a] + grow, Q.gn[a]);
      } else {
        Nlo[a] = ch.blo[a];
        Nhi[a] = ch.bhi[a];
      }
    }
    // Eq. 6-7 between the regions of consecutive iterations
    const Stats sb = box_stats<SW>(Q, prof, nm, lattice_in_box(Q, Nlo, Nhi), sl);
    if (!run) continue;
    const double Wi = sa.scatter + sb.scatter;
    const double pooled = (sa.sum + sb.sum) / static_cast<double>(sa.n + sb.n);
    const double Bi = static_cast<double>(sa.n) * (sa.mean - pooled) * (sa.mean - pooled) +
                      static_cast<double>(sb.n) * (sb.mean - pooled) * (sb.mean - pooled);
    // the stop test; its margin and the metric gap (divisions) are logged
    // after the loop, off this chain of dependent float64 steps
    const bool cont = i < 2 || ((Bi > B_prev) && (Wi < W_prev));
    if (sl == 0) {
      R->child[li] = best;
      R->n_children[li] = nvalid;
      R->metric_top[li] = best_m;
      R->metric_gap[li] = second_m;  // the runner-up until the loop ends
      for (int a = 0; a < 3; ++a) {
        R->box_lo[li][a] = Nlo[a];
        R->box_hi[li][a] = Nhi[a];
      }
      R->within[li] = Wi;
      R->between[li] = Bi;
    }
    n_logged = i;
    if (!cont) {
      stop = UWB_STOP_METRIC;
      iters = i - 1;
      run = false;
      continue;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Rlo[a] = Nlo[a];
      Rhi[a] = Nhi[a];
    }
    sa = sb;
    var_prev = sa.var;
    B_prev = Bi;
    W_prev = Wi;
    iters = i;
    if (i == Q.max_iters) {
      stop = UWB_STOP_CAP;
      run = false;
    }
  }
  // the logged margins, one iteration per lane: every logged iteration after
  // the first followed an accepted one, so B_{i-1} and W_{i-1} are the
  // previous entries
  __syncwarp();
  if (live) {
    for (int li = sl; li < n_logged; li += SW) {
      const double Bi = R->between[li], Wi = R->within[li];
      double margin = 1e300;
      if (li >= 1) {
        const double B_prev = R->between[li - 1], W_prev = R->within[li - 1];
        const double mB = rel_gap(Bi, B_prev), mW = rel_gap(W_prev, Wi);
        margin = (Bi > B_prev) && (Wi < W_prev) ? fmin(mB, mW) : fmax(-mB, -mW);
      }
      R->stop_margin[li] = margin;
      R->metric_gap[li] =
          R->n_children[li] > 1 ? rel_gap(R->metric_top[li], R->metric_gap[li]) : 1e300;
    }
  }
  if (live && sl == 0) {
    R->status = UWB_OK;
    R->iters = iters;
    R->n_logged = n_logged;
    R->stop_reason = stop;
    for (int a = 0; a < 3; ++a) {
      R->roi_lo[a] = Rlo[a];
      R->roi_hi[a] = Rhi[a];
      box->lo[a] = Rlo[a];
      box->step[a] = 1;
      box->cnt[a] = Rhi[a] - Rlo[a];
    }
    box->tiles = lattice_tiles(box->cnt, P.tdim);
  }
}

// ----------------------------------------------- progressive re-evaluation
// A variant of the loop above (the paper's loop reads only the decimated
// profile): from the second iteration on, the child choice -- the variance of
// the region being split (sigma^2_{i-1} of Eq. 5) and the children's Eq. 5
// metrics -- reads a fresh lattice of that region, imaged just before this
// kernel, with at most the decimated lattice's point count per axis (step
// ceil(side / c0), centred). The Eq. 6-7 stopping rule keeps reading the
// decimated profile, so consecutive iterations compare scatters over one
// lattice. Energies are divided by the profile maximum throughout.

// Lattice of the index range [lo, hi) with at most c0 points (first, step, count).
__host__ __device__ inline void region_lattice(int lo, int hi, int c0, int& first, int& step,
                                               int& cnt) {
  const int side = hi - lo;
  int s = (side + c0 - 1) / c0;
  if (s < 1) s = 1;
  const int o = ((side - 1) % s) / 2;
  first = lo + o;
  step = s;
  cnt = (side - 1 - o) / s + 1;
}

__device__ void set_full_box(LatBox* box, const int lo[3], const int hi[3], const int tdim[3]) {
  for (int a = 0; a < 3; ++a) {
    box->lo[a] = lo[a];
    box->step[a] = 1;
    box->cnt[a] = hi[a] - lo[a];
  }
  box->tiles = lattice_tiles(box->cnt, tdim);
}

__device__ void set_empty_box(LatBox* box) {
  for (int a = 0; a < 3; ++a) {
    box->lo[a] = 0;
    box->step[a] = 1;
    box->cnt[a] = 0;
  }
  box->tiles = 0;
}

__global__ void __launch_bounds__(256) k_prog_step(const ProgParams P, int it) {
  const int lane = threadIdx.x & 31;
  const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (s >= P.B) return;
  SelScan Q0;  // the decimated lattice (profile)
  Q0.prof_off = static_cast<long long>(s) * P.stride;
  for (int a = 0; a < 3; ++a) {
    Q0.gn[a] = P.gn[a];
    Q0.off[a] = P.off[a];
    Q0.step[a] = P.step[a];
    Q0.cnt[a] = P.cnt[a];
  }
  Q0.D = P.D;
  Q0.max_iters = P.max_iters;
  const float* prof = P.profile + Q0.prof_off;
  ProgState* S = P.state + s;
  uwb_result* R = P.out + s;
  LatBox* next = P.next_boxes + s;
  LatBox* fin = P.final_boxes + s;
  const int dim = P.dim;
  const long long Pd = static_cast<long long>(Q0.cnt[0]) * Q0.cnt[1] * Q0.cnt[2];

  if (it == 1) {  // the decimated profile: record, maximum, validity
    int* w = reinterpret_cast<int*>(R);
    for (int j = lane; j < static_cast<int>(sizeof(uwb_result) / 4); j += 32) w[j] = 0;
    float fmx = 0.f;
    bool bad = false;
    for (long long j = lane; j < Pd; j += 32) {
      const float v = prof[j];
      bad |= !isfinite(v);
      fmx = fmaxf(fmx, v);
    }
    bad = __any_sync(0xFFFFFFFFu, bad);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fmx = fmaxf(fmx, __shfl_xor_sync(0xFFFFFFFFu, fmx, o));
    __syncwarp();
    if (lane == 0) {
      R->decim = Q0.D;
      for (int a = 0; a < 3; ++a) {
        R->offset[a] = Q0.off[a];
        R->dcount[a] = Q0.cnt[a];
        R->loc_idx[a] = -1;
        S->Rlo[a] = 0;
        S->Rhi[a] = Q0.gn[a];
      }
      R->profile_max = fmx;
      S->pmax = fmx;
      S->B_prev = S->W_prev = 0.0;
      S->points = Pd;
      S->iters = S->n_logged = 0;
      S->stop = UWB_STOP_NONE;
      S->active = !(bad || fmx == 0.f);
      set_empty_box(next);
      if (!S->active) {
        R->status = bad ? UWB_ERR_NONFINITE : UWB_OK;
        R->stop_reason = bad ? UWB_STOP_NONE : UWB_STOP_NO_TARGET;
        set_empty_box(fin);
      }
    }
    __syncwarp();
  }
  if (!S->active) {
    if (lane == 0) set_empty_box(next);
    return;
  }
  const uwb_rule& rule = P.rule;
  const Norm nm = make_norm(S->pmax);
  int Rlo[3], Rhi[3];
  for (int a = 0; a < 3; ++a) {
    Rlo[a] = S->Rlo[a];
    Rhi[a] = S->Rhi[a];
  }
  // the lattice the child choice reads
  SelScan Qc = Q0;
  const float* cv = prof;
  if (it >= 2) {
    for (int a = 0; a < 3; ++a)
      if (a < dim)
        region_lattice(Rlo[a], Rhi[a], Q0.cnt[a], Qc.off[a], Qc.step[a], Qc.cnt[a]);
    cv = P.lattice + Q0.prof_off;
    const long long ni = static_cast<long long>(Qc.cnt[0]) * Qc.cnt[1] * Qc.cnt[2];
    bool bad = false;
    for (long long j = lane; j < ni; j += 32) bad |= !isfinite(cv[j]);
    if (__any_sync(0xFFFFFFFFu, bad)) {
      __syncwarp();
      if (lane == 0) {
        S->active = 0;
        R->status = UWB_ERR_NONFINITE;
        set_empty_box(next);
        set_empty_box(fin);
      }
      return;
    }
  }
  const Stats sr = box_stats<32>(Qc, cv, nm, lattice_in_box(Qc, Rlo, Rhi), lane);
  const double var_prev = sr.var;
  const Choice ch = choose_child<32>(Qc, cv, nm, Rlo, Rhi, dim, rule, var_prev, lane, 0);
  const int best = ch.best, nvalid = ch.nvalid;
  const double best_m = ch.best_m, second_m = ch.second_m;
  int blo[3], bhi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    blo[a] = ch.blo[a];
    bhi[a] = ch.bhi[a];
  }
  const int li = it - 1;
  bool stopped = false;
  int stop = UWB_STOP_NONE, iters = it;
  int Nlo[3] = {0, 0, 0}, Nhi[3] = {0, 0, 0};
  if (nvalid == 0) {
    stopped = true;
    stop = UWB_STOP_MINSIZE;
    iters = it - 1;
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a < dim) {
        const int side = bhi[a] - blo[a];
        const int grow = (side * rule.frame_num + rule.frame_den - 1) / rule.frame_den;
        Nlo[a] = max(blo[a] - grow, 0);
        Nhi[a] = min(bhi[a] + grow, Q0.gn[a]);
      } else {
        Nlo[a] = blo[a];
        Nhi[a] = bhi[a];
      }
    }
    // Eq. 6-7 on the decimated profile between the region and the framed child
    const Stats sa = box_stats<32>(Q0, prof, nm, lattice_in_box(Q0, Rlo, Rhi), lane);
    const Stats sb = box_stats<32>(Q0, prof, nm, lattice_in_box(Q0, Nlo, Nhi), lane);
    const double Wi = sa.scatter + sb.scatter;
    const double pooled = (sa.sum + sb.sum) / static_cast<double>(sa.n + sb.n);
    const double Bi = static_cast<double>(sa.n) * (sa.mean - pooled) * (sa.mean - pooled) +
                      static_cast<double>(sb.n) * (sb.mean - pooled) * (sb.mean - pooled);
    double margin = 1e300;
    bool cont = true;
    if (it >= 2) {
      const double mB = rel_gap(Bi, S->B_prev), mW = rel_gap(S->W_prev, Wi);
      cont = (Bi > S->B_prev) && (Wi < S->W_prev);
      margin = cont ? fmin(mB, mW) : fmax(-mB, -mW);
    }
    __syncwarp();
    if (lane == 0) {
      R->child[li] = best;
      R->n_children[li] = nvalid;
      R->metric_top[li] = best_m;
      R->metric_gap[li] = nvalid > 1 ? rel_gap(best_m, second_m) : 1e300;
      for (int a = 0; a < 3; ++a) {
        R->box_lo[li][a] = Nlo[a];
        R->box_hi[li][a] = Nhi[a];
      }
      R->within[li] = Wi;
      R->between[li] = Bi;
      R->stop_margin[li] = margin;
      S->n_logged = it;
      S->B_prev = Bi;
      S->W_prev = Wi;
    }
    if (!cont) {
      stopped = true;
      stop = UWB_STOP_METRIC;
      iters = it - 1;
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        Rlo[a] = Nlo[a];
        Rhi[a] = Nhi[a];
      }
      if (it == P.max_iters) {
        stopped = true;
        stop = UWB_STOP_CAP;
      }
    }
  }
  __syncwarp();
  if (lane == 0) {
    for (int a = 0; a < 3; ++a) {
      S->Rlo[a] = Rlo[a];
      S->Rhi[a] = Rhi[a];
    }
    S->iters = iters;
    if (stopped) {
      S->active = 0;
      R->status = UWB_OK;
      R->iters = iters;
      R->n_logged = S->n_logged;
      R->stop_reason = stop;
      for (int a = 0; a < 3; ++a) {
        R->roi_lo[a] = Rlo[a];
        R->roi_hi[a] = Rhi[a];
      }
      set_full_box(fin, Rlo, Rhi, P.tdim);
      set_empty_box(next);
    } else {
      // the next iteration's lattice of the new region
      int lo[3], st[3], cn[3];
      long long n = 1;
      for (int a = 0; a < 3; ++a) {
        if (a < dim) {
          region_lattice(Rlo[a], Rhi[a], Q0.cnt[a], lo[a], st[a], cn[a]);
        } else {
          lo[a] = 0;
          st[a] = 1;
          cn[a] = Q0.gn[a];
        }
        n *= cn[a];
      }
      for (int a = 0; a < 3; ++a) {
        next->lo[a] = lo[a];
        next->step[a] = st[a];
        next->cnt[a] = cn[a];
      }
      next->tiles = lattice_tiles(cn, P.tdim);
      S->points += n;
    }
  }
}

// Exclusive prefix sum of the per-scan tile counts (one CTA).
__global__ void __launch_bounds__(1024) k_plan(const LatBox* boxes, int* prefix, int B) {
  __shared__ int warp_tot[32];
  __shared__ int carry_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) carry_s = 0;
  __syncthreads();
  for (int base = 0; base < B; base += blockDim.x) {
    const int idx = base + tid;
    const int v = idx < B ? boxes[idx].tiles : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const int nw = blockDim.x >> 5;
      int w = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xFFFFFFFFu, w, o);
        if (lane >= o) w += u;
      }
      if (lane < nw) warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const int carry = carry_s;
    const int before = (warp > 0 ? warp_tot[warp - 1] : 0) + incl - v;
    if (idx < B) prefix[idx] = carry + before;
    __syncthreads();
    if (tid == 0) carry_s = carry + warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
  }
  if (tid == 0) prefix[B] = carry_s;
}

// Decodes each scan's argmax key into the result record.
__global__ void k_finish(const FinishParams P, const int* status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.B) return;
  FinScan F;
  if (P.scans) {
    F = P.scans[s];
  } else {
    for (int a = 0; a < 3; ++a) {
      F.gn[a] = P.gn[a];
      F.org[a] = P.org[a];
      F.pit[a] = P.pit[a];
    }
    F.Pd = P.Pd;
  }
  uwb_result* R = P.out + s;
  const LatBox b = P.boxes[s];
  const unsigned long long key = P.keys[s];
  const long long roi = b.tiles > 0 ? static_cast<long long>(b.cnt[0]) * b.cnt[1] * b.cnt[2] : 0;
  R->points_evaluated = F.Pd + roi;
  if (P.learn)  // learned localisation: coarse maps, plus the profile where Eq. 5 decided
    R->points_evaluated = (P.learn[s].fallback ? F.Pd : 0) + P.learn[s].map_points + roi;
  if (P.prog)  // progressive loop: the profile and every region lattice imaged
    R->points_evaluated = P.prog[s].points + roi;
  if (status && *status != UWB_OK) R->status = *status;
  if (key != 0ull && b.tiles > 0) {
    const long long lin = static_cast<long long>(0xFFFFFFFFull - (key & 0xFFFFFFFFull));
    const int ix = static_cast<int>(lin % F.gn[0]);
    const int iy = static_cast<int>((lin / F.gn[0]) % F.gn[1]);
    const int iz = static_cast<int>(lin / (static_cast<long long>(F.gn[0]) * F.gn[1]));
    const int idx[3] = {ix, iy, iz};
    for (int a = 0; a < 3; ++a) {
      R->loc_idx[a] = idx[a];
      R->loc_xyz[a] = F.org[a] + static_cast<double>(idx[a]) * F.pit[a];
    }
    R->peak = static_cast<double>(__uint_as_float(static_cast<unsigned int>(key >> 32)));
  } else {
    for (int a = 0; a < 3; ++a) {
      R->loc_idx[a] = -1;
      R->loc_xyz[a] = 0.0;
    }
    R->peak = 0.0;
  }
}

// Tumour-presence verdict per scan: both runs located the same focal point.
__global__ void k_presence(const uwb_result* a, const uwb_result* b, int* present, int B) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  const uwb_result& x = a[s];
  const uwb_result& y = b[s];
  int same = x.status == UWB_OK && y.status == UWB_OK && x.loc_idx[0] >= 0 && y.loc_idx[0] >= 0;
  for (int k = 0; k < 3; ++k) same = same && x.loc_idx[k] == y.loc_idx[k];
  present[s] = same;
}

// argmax keys -> linear index (or -1), in place.
__global__ void k_keys_to_index(unsigned long long* keys, int B) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  const unsigned long long key = keys[s];
  const long long idx =
      key ? static_cast<long long>(0xFFFFFFFFull - (key & 0xFFFFFFFFull)) : -1ll;
  reinterpret_cast<long long*>(keys)[s] = idx;
}

}  // namespace

// Four scans per warp for large uniform batches of small profiles (a lane's
// share of a scan's points stays short); otherwise a warp per scan. Packed
// warps run as CTAs of one warp, so that the few warps of a batch spread
// evenly over the SMs.
cudaError_t launch_select(const SelParams& p, cudaStream_t st) {
  const long long Pd = static_cast<long long>(p.cnt[0]) * p.cnt[1] * p.cnt[2];
  if (!p.scans && p.B >= kSelectPackedMinScans && Pd <= kSelectPackedMaxPoints) {
    k_select<8><<<(p.B + 3) / 4, 32, 0, st>>>(p);
  } else {
    const int warps = 8;
    k_select<32><<<(p.B + warps - 1) / warps, warps * 32, 0, st>>>(p);
  }
  return cudaGetLastError();
}

cudaError_t launch_plan(const LatBox* boxes, int* prefix, int B, cudaStream_t st) {
  k_plan<<<1, 1024, 0, st>>>(boxes, prefix, B);
  return cudaGetLastError();
}

cudaError_t launch_prog_step(const ProgParams& p, int iteration, cudaStream_t st) {
  k_prog_step<<<(p.B + 7) / 8, 256, 0, st>>>(p, iteration);
  return cudaGetLastError();
}

cudaError_t launch_finish(const FinishParams& p, const int* status, cudaStream_t st) {
  k_finish<<<(p.B + 127) / 128, 128, 0, st>>>(p, status);
  return cudaGetLastError();
}

cudaError_t launch_presence(const uwb_result* a, const uwb_result* b, int* present, int B,
                            cudaStream_t st) {
  k_presence<<<(B + 127) / 128, 128, 0, st>>>(a, b, present, B);
  return cudaGetLastError();
}

cudaError_t launch_keys_to_index(unsigned long long* keys, int B, cudaStream_t st) {
  k_keys_to_index<<<(B + 127) / 128, 128, 0, st>>>(keys, B);
  return cudaGetLastError();
}

}  // namespace uwb
