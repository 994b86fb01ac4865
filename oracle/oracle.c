/*
 * FP64 CPU oracle for segment-search confocal UWB imaging (arXiv:1709.02549).
 *
 * TEST INFRASTRUCTURE: used only by the test suite, the smoke check and the
 * benchmark's CPU-baseline leg. It shares no code with the CUDA library.
 *
 * Readings of the paper that this file fixes (the paper is silent or garbled
 * there):
 *  - Eq. 1 prints |r - r_iT| / (2 c dt); the round trip of a monostatic echo
 *    is read as tau_i = 2 |r - a_i| / v with v = c / sqrt(eps_r), and the
 *    delay in samples is u_i = tau_i * fs.
 *  - Eq. 3 sums Y_i(t - n_i(r)) over a time window; the aligned signal is read
 *    as x_i(k) = Y_i(u_i - h + k), k = 0 .. W-1, h = floor(W/2), a window
 *    centred on the delay. Fractional delays use linear interpolation between
 *    the two neighbouring samples; samples outside [0, N-1] are zero.
 *  - DMAS (Section II.B) multiplies every pair of aligned signals (i < j) and
 *    sums the products; that sum is squared and summed over the window, as
 *    DAS's sum is in Eq. 3. No sign-preserving square root is applied.
 *  - Eq. 5 mixes the units of the mean and the variance; the decimated
 *    energies are divided by their maximum before any metric is taken, so
 *    scaling the traces changes no decision.
 *  - sigma^2_{i-1} in Eq. 5 is the variance of the region being split (the
 *    whole region at the first iteration); variances are population (1/N).
 *    A child with zero variance has metric = its mean.
 *  - The two "classes" of Eq. 6-7 are the decimated energies of the regions
 *    of two consecutive iterations (R_{i-1}, R_i), each scalar; the pooled
 *    mean is over both. The loop continues while B grows and W shrinks,
 *    tested from the second iteration; on failure the last accepted region
 *    R_{i-1} is the result.
 *  - Sliding framing: each iteration's chosen child grows by
 *    ceil(frame_num/frame_den * side) points on each side, clipped to the grid.
 *  - Children with no decimated point, or with a side shorter than
 *    min_segment points, are not candidates. Ties go to the lowest child
 *    index (z, then y, then x; low half first) and to the lowest linear
 *    focal-point index (x fastest).
 *  - The decimated lattice along an axis of n points is {o + D k} with
 *    o = ((n - 1) mod D) / 2, which centres it.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Y_i[n], zero outside the recorded trace. */
static double trace_sample(const float* row, int N, long n) {
  if (n < 0 || n >= N) return 0.0;
  return (double)row[n];
}

/* Energy of one focal point r (Eq. 1 + Eq. 3, or Eq. 1 + DMAS). u and x are
 * caller scratch of M doubles each. */
static double focal_energy(const float* traces, int M, int N, const float* ant,
                           const double r[3], double v, double fs, int W, int bf,
                           double* u, double* x) {
  const int h = W / 2;
  for (int i = 0; i < M; ++i) {
    double dx = r[0] - (double)ant[3 * i + 0];
    double dy = r[1] - (double)ant[3 * i + 1];
    double dz = r[2] - (double)ant[3 * i + 2];
    double dist = sqrt(dx * dx + dy * dy + dz * dz);
    u[i] = 2.0 * dist / v * fs; /* round-trip delay in samples */
  }
  double energy = 0.0;
  for (int k = 0; k < W; ++k) {
    for (int i = 0; i < M; ++i) {
      double t = u[i] - (double)h + (double)k;
      double n0 = floor(t);
      double f = t - n0;
      const float* row = traces + (size_t)i * (size_t)N;
      x[i] = (1.0 - f) * trace_sample(row, N, (long)n0) +
             f * trace_sample(row, N, (long)n0 + 1);
    }
    double s = 0.0;
    if (bf == ORC_DAS) {
      for (int i = 0; i < M; ++i) s += x[i];
    } else {
      for (int i = 0; i < M; ++i)
        for (int j = i + 1; j < M; ++j) s += x[i] * x[j];
    }
    energy += s * s;
  }
  return energy;
}

int orc_image(const float* traces, int M, int N, const float* antennas,
              const orc_grid* g, double v, double fs, int window, int beamformer,
              const int lo[3], const int step[3], const int cnt[3], double* out) {
  if (!traces || !antennas || !g || !out || M < 1 || N < 1 || window < 1 ||
      !(v > 0) || !(fs > 0) || (beamformer != ORC_DAS && beamformer != ORC_DMAS))
    return ORC_ERR_ARG;
  const long long total = (long long)cnt[0] * cnt[1] * cnt[2];
  int bad = 0;
#pragma omp parallel
  {
    double* u = (double*)malloc(sizeof(double) * (size_t)M);
    double* x = (double*)malloc(sizeof(double) * (size_t)M);
    if (!u || !x) {
#pragma omp atomic write
      bad = 1;
    } else {
#pragma omp for schedule(dynamic, 16)
      for (long long p = 0; p < total; ++p) {
        long long kx = p % cnt[0];
        long long ky = (p / cnt[0]) % cnt[1];
        long long kz = p / ((long long)cnt[0] * cnt[1]);
        long long kk[3] = {kx, ky, kz};
        double r[3];
        for (int a = 0; a < 3; ++a) {
          long long idx = lo[a] + step[a] * kk[a];
          r[a] = g->origin[a] + (double)idx * g->pitch[a];
        }
        out[p] = focal_energy(traces, M, N, antennas, r, v, fs, window, beamformer,
                              u, x);
      }
    }
    free(u);
    free(x);
  }
  return bad ? ORC_ERR_ARG : ORC_OK;
}

/* Multistatic energy of one focal point (Eq. 2 + Eq. 4, or Eq. 2 + DMAS over
 * channel pairs). u and x are caller scratch of C doubles each. */
static double focal_energy_ms(const float* traces, int C, int N, const int* chan,
                              const float* ant, const double r[3], double v, double fs, int W,
                              int bf, double* u, double* x) {
  const int h = W / 2;
  for (int c = 0; c < C; ++c) {
    double path = 0.0;
    for (int e = 0; e < 2; ++e) {
      const int i = chan[2 * c + e];
      double dx = r[0] - (double)ant[3 * i + 0];
      double dy = r[1] - (double)ant[3 * i + 1];
      double dz = r[2] - (double)ant[3 * i + 2];
      path += sqrt(dx * dx + dy * dy + dz * dz);
    }
    u[c] = path / v * fs; /* transmitter -> focal point -> receiver, in samples */
  }
  double energy = 0.0;
  for (int k = 0; k < W; ++k) {
    for (int c = 0; c < C; ++c) {
      double t = u[c] - (double)h + (double)k;
      double n0 = floor(t);
      double f = t - n0;
      const float* row = traces + (size_t)c * (size_t)N;
      x[c] = (1.0 - f) * trace_sample(row, N, (long)n0) +
             f * trace_sample(row, N, (long)n0 + 1);
    }
    double s = 0.0;
    if (bf == ORC_DAS) {
      for (int c = 0; c < C; ++c) s += x[c];
    } else {
      for (int c = 0; c < C; ++c)
        for (int d = c + 1; d < C; ++d) s += x[c] * x[d];
    }
    energy += s * s;
  }
  return energy;
}

int orc_image_multistatic(const float* traces, int C, int N, const int* chan,
                          const float* antennas, int M, const orc_grid* g, double v, double fs,
                          int window, int beamformer, const int lo[3], const int step[3],
                          const int cnt[3], double* out) {
  if (!traces || !chan || !antennas || !g || !out || C < 1 || N < 1 || M < 1 || window < 1 ||
      !(v > 0) || !(fs > 0) || (beamformer != ORC_DAS && beamformer != ORC_DMAS))
    return ORC_ERR_ARG;
  for (int c = 0; c < 2 * C; ++c)
    if (chan[c] < 0 || chan[c] >= M) return ORC_ERR_ARG;
  const long long total = (long long)cnt[0] * cnt[1] * cnt[2];
  int bad = 0;
#pragma omp parallel
  {
    double* u = (double*)malloc(sizeof(double) * (size_t)C);
    double* x = (double*)malloc(sizeof(double) * (size_t)C);
    if (!u || !x) {
#pragma omp atomic write
      bad = 1;
    } else {
#pragma omp for schedule(dynamic, 16)
      for (long long p = 0; p < total; ++p) {
        long long kk[3] = {p % cnt[0], (p / cnt[0]) % cnt[1], p / ((long long)cnt[0] * cnt[1])};
        double r[3];
        for (int a = 0; a < 3; ++a)
          r[a] = g->origin[a] + (double)(lo[a] + step[a] * kk[a]) * g->pitch[a];
        out[p] = focal_energy_ms(traces, C, N, chan, antennas, r, v, fs, window, beamformer, u,
                                 x);
      }
    }
    free(u);
    free(x);
  }
  return bad ? ORC_ERR_ARG : ORC_OK;
}

/* Section III: manual mode takes D as given; automatic mode spaces samples
 * by the side of the square inscribed in the smallest tumour to be detected
 * (d / sqrt 2), in units of the final resolution (Section IV: 1 cm and 1 mm
 * give D = 7). */
int orc_decimation(const orc_rule* r, const orc_grid* g) {
  if (r->mode == ORC_DECIM_MANUAL) return r->decimation >= 1 ? r->decimation : 1;
  double res = g->pitch[0];
  for (int a = 1; a < g->dim; ++a)
    if (g->pitch[a] < res) res = g->pitch[a];
  double side = r->min_tumor_diameter / sqrt(2.0);
  int D = (int)floor(side / res + 1e-9);
  return D < 1 ? 1 : D;
}

int orc_lattice_offset(int n, int D) { return ((n - 1) % D) / 2; }

/* ---------------------------------------------------------------- selection */

typedef struct {
  int dim;
  int n[3];
  int off[3], step[3], cnt[3];
} lattice;

static void make_lattice(const orc_grid* g, int D, lattice* L) {
  L->dim = g->dim;
  for (int a = 0; a < 3; ++a) {
    L->n[a] = g->n[a];
    if (a < g->dim) {
      L->off[a] = orc_lattice_offset(g->n[a], D);
      L->step[a] = D;
      L->cnt[a] = (g->n[a] - 1 - L->off[a]) / D + 1;
    } else {
      L->off[a] = 0;
      L->step[a] = 1;
      L->cnt[a] = g->n[a];
    }
  }
}

/* Copies the decimated energies that fall in box [lo, hi) into buf; returns
 * how many. Plain scan over every decimated point. */
static long gather_box(const double* e, const lattice* L, const int lo[3],
                       const int hi[3], double* buf) {
  long n = 0;
  for (int kz = 0; kz < L->cnt[2]; ++kz)
    for (int ky = 0; ky < L->cnt[1]; ++ky)
      for (int kx = 0; kx < L->cnt[0]; ++kx) {
        int idx[3] = {L->off[0] + L->step[0] * kx, L->off[1] + L->step[1] * ky,
                      L->off[2] + L->step[2] * kz};
        int in = 1;
        for (int a = 0; a < 3; ++a)
          if (idx[a] < lo[a] || idx[a] >= hi[a]) in = 0;
        if (in) buf[n++] = e[kx + (long)L->cnt[0] * (ky + (long)L->cnt[1] * kz)];
      }
  return n;
}

static double mean_of(const double* x, long n) {
  double s = 0.0;
  for (long i = 0; i < n; ++i) s += x[i];
  return s / (double)n;
}

static double var_of(const double* x, long n) {
  double m = mean_of(x, n);
  double s = 0.0;
  for (long i = 0; i < n; ++i) s += (x[i] - m) * (x[i] - m);
  return s / (double)n;
}

/* Eq. 5: M_i = (1 - a) mu_i + a sigma_i^2, a = (sigma_i^2 - sigma_{i-1}^2) / sigma_i^2.
 * The paper describes a as the weight that moves the metric from the mean
 * (equal variances) to the variance (distinct variances); read as a convex
 * weight it is clipped to [0, 1]. clip = 0 evaluates the printed formula
 * with no clipping. */
static double hybrid(double mean_i, double var_i, double var_prev, int clip) {
  if (var_i == 0.0) return mean_i;
  double a = (var_i - var_prev) / var_i;
  if (clip) a = a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
  return (1.0 - a) * mean_i + a * var_i;
}

double orc_hybrid_metric(double mean_i, double var_i, double var_prev) {
  return hybrid(mean_i, var_i, var_prev, 1);
}

double orc_hybrid_metric_unclipped(double mean_i, double var_i, double var_prev) {
  return hybrid(mean_i, var_i, var_prev, 0);
}

/* Eq. 6 (within-class scatter) and Eq. 7 (between-class scatter) for two
 * classes of scalars. */
void orc_scatter(const double* a, int na, const double* b, int nb, double* within,
                 double* between) {
  double ma = mean_of(a, na), mb = mean_of(b, nb);
  double w = 0.0;
  for (int i = 0; i < na; ++i) w += (a[i] - ma) * (a[i] - ma);
  for (int i = 0; i < nb; ++i) w += (b[i] - mb) * (b[i] - mb);
  double tot = 0.0;
  for (int i = 0; i < na; ++i) tot += a[i];
  for (int i = 0; i < nb; ++i) tot += b[i];
  double m = tot / (double)(na + nb);
  *within = w;
  *between = (double)na * (ma - m) * (ma - m) + (double)nb * (mb - m) * (mb - m);
}

static int default_iters(const orc_grid* g) {
  int nmax = 1;
  for (int a = 0; a < g->dim; ++a)
    if (g->n[a] > nmax) nmax = g->n[a];
  int lg = 0;
  while ((1 << lg) < nmax) ++lg;
  return lg + 2;
}

static double rel_gap(double hi, double lo) {
  double d = fabs(hi) > fabs(lo) ? fabs(hi) : fabs(lo);
  if (d == 0.0) return 0.0;
  return (hi - lo) / d;
}

/* Test aid (orc_path): clears the path's outputs. */
static void path_reset(orc_path* p) {
  if (!p) return;
  p->error = 0;
  for (int i = 0; i < ORC_MAX_ITERS; ++i) {
    p->own_child[i] = -1;
    p->own_cont[i] = -1;
    p->taken_metric[i] = 0.0;
    p->taken_gap[i] = 0.0;
  }
}

/* Test aid (orc_path): the child iteration li + 1 takes, the path's if it
 * names one, else the argmax `best`; -1 if the path names a non-candidate. */
static int path_take_child(orc_path* p, int li, int nchild, int best, double best_m,
                           const int* valid, const double* metric) {
  int take = best;
  if (p && li < p->n && p->child[li] >= 0) {
    take = p->child[li];
    if (take >= nchild || !valid[take]) {
      p->error = li + 1;
      return -1;
    }
  }
  if (p) {
    p->own_child[li] = best;
    p->taken_metric[li] = metric[take];
    p->taken_gap[li] = take == best ? 0.0 : rel_gap(best_m, metric[take]);
  }
  return take;
}

/* Test aid (orc_path): the continue (1) / stop (0) outcome iteration li + 1
 * takes, the path's if it names one, else the Eq. 6-7 test's `cont`. */
static int path_take_cont(orc_path* p, int li, int cont) {
  if (!p) return cont;
  p->own_cont[li] = cont;
  if (li < p->n && p->cont[li] >= 0) return p->cont[li] ? 1 : 0;
  return cont;
}

int orc_select(const double* e, const orc_grid* g, const orc_rule* r, int D,
               orc_result* res) {
  return orc_select_path(e, g, r, D, NULL, res);
}

int orc_select_path(const double* e, const orc_grid* g, const orc_rule* r, int D,
                    orc_path* path, orc_result* res) {
  path_reset(path);
  lattice L;
  make_lattice(g, D, &L);
  const long total = (long)L.cnt[0] * L.cnt[1] * L.cnt[2];
  double* bufa = (double*)malloc(sizeof(double) * (size_t)total);
  double* bufb = (double*)malloc(sizeof(double) * (size_t)total);
  double* bufc = (double*)malloc(sizeof(double) * (size_t)total);
  if (!bufa || !bufb || !bufc) {
    free(bufa); free(bufb); free(bufc);
    return ORC_ERR_ARG;
  }
  int max_iters = r->max_iters > 0 ? r->max_iters : default_iters(g);
  if (max_iters > ORC_MAX_ITERS) max_iters = ORC_MAX_ITERS;
  const int nchild = 1 << g->dim;

  int R_lo[3] = {0, 0, 0}, R_hi[3] = {g->n[0], g->n[1], g->n[2]};
  long na = gather_box(e, &L, R_lo, R_hi, bufa);
  double var_prev = var_of(bufa, na); /* whole region at the first iteration */
  double B_prev = 0.0, W_prev = 0.0;
  res->stop_reason = ORC_STOP_NONE;
  res->iters = 0;
  res->n_logged = 0;

  for (int i = 1; i <= max_iters; ++i) {
    const int li = i - 1;
    int mid[3];
    for (int a = 0; a < 3; ++a) mid[a] = R_lo[a] + (R_hi[a] - R_lo[a]) / 2;

    int best = -1, nvalid = 0;
    double best_m = 0.0, second_m = 0.0;
    int clo[8][3], chi[8][3], valid[8] = {0};
    double metric[8] = {0};
    for (int c = 0; c < nchild; ++c) {
      int ok = 1;
      for (int a = 0; a < 3; ++a) {
        if (a < g->dim) {
          int bit = (c >> a) & 1; /* x is bit 0, y bit 1, z bit 2 */
          clo[c][a] = bit ? mid[a] : R_lo[a];
          chi[c][a] = bit ? R_hi[a] : mid[a];
          if (chi[c][a] - clo[c][a] < r->min_segment) ok = 0;
        } else {
          clo[c][a] = R_lo[a];
          chi[c][a] = R_hi[a];
        }
      }
      if (!ok) continue;
      long nc = gather_box(e, &L, clo[c], chi[c], bufc);
      if (nc == 0) continue;
      double mu = mean_of(bufc, nc), var = var_of(bufc, nc);
      double m;
      if (r->metric == ORC_METRIC_MEAN)
        m = mu;
      else if (r->metric == ORC_METRIC_VARIANCE)
        m = var;
      else if (r->metric == ORC_METRIC_HYBRID_UNCLIPPED)
        m = orc_hybrid_metric_unclipped(mu, var, var_prev);
      else
        m = orc_hybrid_metric(mu, var, var_prev);
      valid[c] = 1;
      metric[c] = m;
      if (nvalid == 0 || m > best_m) {
        if (nvalid > 0) second_m = best_m;
        best_m = m;
        best = c;
      } else if (nvalid == 1 || m > second_m) {
        second_m = m;
      }
      ++nvalid;
    }
    if (nvalid == 0) {
      res->stop_reason = ORC_STOP_MINSIZE;
      res->iters = i - 1;
      break;
    }
    const int take = path_take_child(path, li, nchild, best, best_m, valid, metric);
    if (take < 0) {
      free(bufa); free(bufb); free(bufc);
      return ORC_ERR_ARG;
    }
    const int* best_lo = clo[take];
    const int* best_hi = chi[take];
    res->child[li] = take;
    res->n_children[li] = nvalid;
    res->metric_top[li] = metric[take];
    res->metric_gap[li] = nvalid > 1 ? rel_gap(best_m, second_m) : 1e300;

    /* sliding framing of the chosen child */
    int N_lo[3], N_hi[3];
    for (int a = 0; a < 3; ++a) {
      if (a < g->dim) {
        int side = best_hi[a] - best_lo[a];
        int grow = (side * r->frame_num + r->frame_den - 1) / r->frame_den;
        N_lo[a] = best_lo[a] - grow < 0 ? 0 : best_lo[a] - grow;
        N_hi[a] = best_hi[a] + grow > g->n[a] ? g->n[a] : best_hi[a] + grow;
      } else {
        N_lo[a] = best_lo[a];
        N_hi[a] = best_hi[a];
      }
      res->box_lo[li][a] = N_lo[a];
      res->box_hi[li][a] = N_hi[a];
    }

    /* Eq. 6-7 between the regions of two consecutive iterations */
    long nb = gather_box(e, &L, N_lo, N_hi, bufb);
    double Wi, Bi;
    orc_scatter(bufa, (int)na, bufb, (int)nb, &Wi, &Bi);
    res->within[li] = Wi;
    res->between[li] = Bi;
    res->n_logged = i;
    if (i >= 2) {
      double mB = rel_gap(Bi, B_prev);  /* > 0: B grew */
      double mW = rel_gap(W_prev, Wi);  /* > 0: W shrank */
      int cont = (Bi > B_prev) && (Wi < W_prev);
      res->stop_margin[li] = cont ? (mB < mW ? mB : mW) : (-mB > -mW ? -mB : -mW);
      if (!path_take_cont(path, li, cont)) {
        res->stop_reason = ORC_STOP_METRIC;
        res->iters = i - 1;
        break;
      }
    } else {
      res->stop_margin[li] = 1e300;
    }
    memcpy(R_lo, N_lo, sizeof N_lo);
    memcpy(R_hi, N_hi, sizeof N_hi);
    memcpy(bufa, bufb, sizeof(double) * (size_t)nb);
    na = nb;
    var_prev = var_of(bufa, na);
    B_prev = Bi;
    W_prev = Wi;
    res->iters = i;
    if (i == max_iters) {
      res->stop_reason = ORC_STOP_CAP;
      break;
    }
  }
  for (int a = 0; a < 3; ++a) {
    res->roi_lo[a] = R_lo[a];
    res->roi_hi[a] = R_hi[a];
  }
  free(bufa);
  free(bufb);
  free(bufc);
  return ORC_OK;
}

/* The data a localisation images: monostatic (chan == NULL, rows = antennas)
 * or multistatic (rows = channels). */
typedef struct {
  const float* traces;
  int rows, N;
  const int* chan;
  const float* antennas;
  int M;
  double v, fs;
  int window, beamformer;
} scan_data;

static int scan_image(const scan_data* d, const orc_grid* g, const int lo[3], const int step[3],
                      const int cnt[3], double* out) {
  if (d->chan)
    return orc_image_multistatic(d->traces, d->rows, d->N, d->chan, d->antennas, d->M, g, d->v,
                                 d->fs, d->window, d->beamformer, lo, step, cnt, out);
  return orc_image(d->traces, d->rows, d->N, d->antennas, g, d->v, d->fs, d->window,
                   d->beamformer, lo, step, cnt, out);
}

static int localize_data(const scan_data* d, const orc_grid* g, const orc_rule* r,
                         orc_path* path, orc_result* res);

int orc_localize(const float* traces, int M, int N, const float* antennas,
                 const orc_grid* g, double v, double fs, int window, int beamformer,
                 const orc_rule* r, orc_result* res) {
  return orc_localize_path(traces, M, N, antennas, g, v, fs, window, beamformer, r, NULL, res);
}

int orc_localize_path(const float* traces, int M, int N, const float* antennas,
                      const orc_grid* g, double v, double fs, int window, int beamformer,
                      const orc_rule* r, orc_path* path, orc_result* res) {
  scan_data d = {traces, M, N, NULL, antennas, M, v, fs, window, beamformer};
  return localize_data(&d, g, r, path, res);
}

int orc_localize_multistatic(const float* traces, int C, int N, const int* chan,
                             const float* antennas, int M, const orc_grid* g, double v,
                             double fs, int window, int beamformer, const orc_rule* r,
                             orc_result* res) {
  return orc_localize_multistatic_path(traces, C, N, chan, antennas, M, g, v, fs, window,
                                       beamformer, r, NULL, res);
}

int orc_localize_multistatic_path(const float* traces, int C, int N, const int* chan,
                                  const float* antennas, int M, const orc_grid* g, double v,
                                  double fs, int window, int beamformer, const orc_rule* r,
                                  orc_path* path, orc_result* res) {
  scan_data d = {traces, C, N, chan, antennas, M, v, fs, window, beamformer};
  return localize_data(&d, g, r, path, res);
}

static int localize_data(const scan_data* d, const orc_grid* g, const orc_rule* r,
                         orc_path* path, orc_result* res) {
  path_reset(path);
  memset(res, 0, sizeof *res);
  for (int a = 0; a < 3; ++a) res->loc_idx[a] = -1;
  if (!g || !r || g->dim < 2 || g->dim > 3 || (g->dim == 2 && g->n[2] != 1) ||
      r->frame_den < 1 || r->frame_num < 0 || r->min_segment < 1) {
    res->status = ORC_ERR_ARG;
    return ORC_ERR_ARG;
  }
  const int D = orc_decimation(r, g);
  lattice L;
  make_lattice(g, D, &L);
  res->decim = D;
  for (int a = 0; a < 3; ++a) {
    res->offset[a] = L.off[a];
    res->dcount[a] = L.cnt[a];
  }
  const long long nd = (long long)L.cnt[0] * L.cnt[1] * L.cnt[2];
  double* prof = (double*)malloc(sizeof(double) * (size_t)nd);
  if (!prof) {
    res->status = ORC_ERR_ARG;
    return ORC_ERR_ARG;
  }
  int st = scan_image(d, g, L.off, L.step, L.cnt, prof);
  if (st != ORC_OK) {
    free(prof);
    res->status = st;
    return st;
  }
  res->points_evaluated = nd;
  double mx = 0.0;
  for (long long p = 0; p < nd; ++p) {
    if (!isfinite(prof[p])) {
      free(prof);
      res->status = ORC_ERR_NONFINITE;
      return ORC_ERR_NONFINITE;
    }
    if (prof[p] > mx) mx = prof[p];
  }
  res->profile_max = mx;
  if (mx == 0.0) {
    free(prof);
    res->stop_reason = ORC_STOP_NO_TARGET;
    return ORC_OK;
  }
  for (long long p = 0; p < nd; ++p) prof[p] /= mx; /* normalised energies */
  st = orc_select_path(prof, g, r, D, path, res);
  free(prof);
  if (st != ORC_OK) {
    res->status = st;
    return st;
  }

  /* final imaging of the region at full resolution, then its argmax */
  int step1[3] = {1, 1, 1}, cnt[3];
  for (int a = 0; a < 3; ++a) cnt[a] = res->roi_hi[a] - res->roi_lo[a];
  const long long nr = (long long)cnt[0] * cnt[1] * cnt[2];
  double* img = (double*)malloc(sizeof(double) * (size_t)(nr > 0 ? nr : 1));
  if (!img) {
    res->status = ORC_ERR_ARG;
    return ORC_ERR_ARG;
  }
  st = scan_image(d, g, res->roi_lo, step1, cnt, img);
  if (st != ORC_OK) {
    free(img);
    res->status = st;
    return st;
  }
  res->points_evaluated += nr;
  long long best = -1;
  for (long long p = 0; p < nr; ++p)
    if (best < 0 || img[p] > img[best]) best = p;
  if (best >= 0) {
    long long k[3] = {best % cnt[0], (best / cnt[0]) % cnt[1],
                      best / ((long long)cnt[0] * cnt[1])};
    for (int a = 0; a < 3; ++a) {
      res->loc_idx[a] = res->roi_lo[a] + (int)k[a];
      res->loc_xyz[a] = g->origin[a] + (double)res->loc_idx[a] * g->pitch[a];
    }
    res->peak = img[best];
  }
  free(img);
  return ORC_OK;
}

/* ------------------------------------------------- progressive re-evaluation */

void orc_region_lattice(int lo, int hi, int c0, int* first, int* step, int* cnt) {
  const int side = hi - lo;
  int s = (side + c0 - 1) / c0;
  if (s < 1) s = 1;
  const int o = ((side - 1) % s) / 2;
  *first = lo + o;
  *step = s;
  *cnt = (side - 1 - o) / s + 1;
}

int orc_localize_progressive(const float* traces, int M, int N, const float* antennas,
                             const orc_grid* g, double v, double fs, int window,
                             int beamformer, const orc_rule* r, orc_result* res) {
  return orc_localize_progressive_path(traces, M, N, antennas, g, v, fs, window, beamformer, r,
                                       NULL, res);
}

int orc_localize_progressive_path(const float* traces, int M, int N, const float* antennas,
                                  const orc_grid* g, double v, double fs, int window,
                                  int beamformer, const orc_rule* r, orc_path* path,
                                  orc_result* res) {
  scan_data d = {traces, M, N, NULL, antennas, M, v, fs, window, beamformer};
  path_reset(path);
  memset(res, 0, sizeof *res);
  for (int a = 0; a < 3; ++a) res->loc_idx[a] = -1;
  if (!g || !r || g->dim < 2 || g->dim > 3 || (g->dim == 2 && g->n[2] != 1) ||
      r->frame_den < 1 || r->frame_num < 0 || r->min_segment < 1) {
    res->status = ORC_ERR_ARG;
    return ORC_ERR_ARG;
  }
  const int D = orc_decimation(r, g);
  lattice L0, L;
  make_lattice(g, D, &L0);
  res->decim = D;
  for (int a = 0; a < 3; ++a) {
    res->offset[a] = L0.off[a];
    res->dcount[a] = L0.cnt[a];
  }
  const long nd = (long)L0.cnt[0] * L0.cnt[1] * L0.cnt[2];
  double* prof = (double*)malloc(sizeof(double) * (size_t)nd);
  double* e = (double*)malloc(sizeof(double) * (size_t)nd);
  double* bufa = (double*)malloc(sizeof(double) * (size_t)nd);
  double* bufb = (double*)malloc(sizeof(double) * (size_t)nd);
  double* bufc = (double*)malloc(sizeof(double) * (size_t)nd);
  if (!prof || !e || !bufa || !bufb || !bufc) {
    free(prof); free(e); free(bufa); free(bufb); free(bufc);
    res->status = ORC_ERR_ARG;
    return ORC_ERR_ARG;
  }
  int st = scan_image(&d, g, L0.off, L0.step, L0.cnt, prof);
  double pmax = 0.0;
  if (st == ORC_OK)
    for (long p = 0; p < nd; ++p) {
      if (!isfinite(prof[p])) st = ORC_ERR_NONFINITE;
      else if (prof[p] > pmax) pmax = prof[p];
    }
  res->points_evaluated = nd;
  res->profile_max = pmax;
  if (st != ORC_OK || pmax == 0.0) {
    free(prof); free(e); free(bufa); free(bufb); free(bufc);
    res->status = st;
    if (st == ORC_OK) res->stop_reason = ORC_STOP_NO_TARGET;
    return st;
  }
  for (long p = 0; p < nd; ++p) prof[p] /= pmax;

  int max_iters = r->max_iters > 0 ? r->max_iters : default_iters(g);
  if (max_iters > ORC_MAX_ITERS) max_iters = ORC_MAX_ITERS;
  const int nchild = 1 << g->dim;
  int R_lo[3] = {0, 0, 0}, R_hi[3] = {g->n[0], g->n[1], g->n[2]};
  long na = gather_box(prof, &L0, R_lo, R_hi, bufa); /* Eq. 6-7 class of R (profile) */
  double B_prev = 0.0, W_prev = 0.0;
  res->stop_reason = ORC_STOP_NONE;

  for (int i = 1; i <= max_iters; ++i) {
    const int li = i - 1;
    /* the lattice the child choice reads: the profile at iteration 1, then
     * the region being split imaged again on its own lattice */
    const double* ce = prof;
    L = L0;
    if (i >= 2) {
      for (int a = 0; a < 3; ++a) {
        if (a < g->dim) {
          orc_region_lattice(R_lo[a], R_hi[a], L0.cnt[a], &L.off[a], &L.step[a], &L.cnt[a]);
        } else {
          L.off[a] = 0;
          L.step[a] = 1;
          L.cnt[a] = g->n[a];
        }
      }
      const long ni = (long)L.cnt[0] * L.cnt[1] * L.cnt[2];
      st = scan_image(&d, g, L.off, L.step, L.cnt, e);
      for (long p = 0; st == ORC_OK && p < ni; ++p)
        if (!isfinite(e[p])) st = ORC_ERR_NONFINITE;
      if (st != ORC_OK) break;
      for (long p = 0; p < ni; ++p) e[p] /= pmax;
      res->points_evaluated += ni;
      ce = e;
    }
    /* sigma^2_{i-1} of Eq. 5: the region being split, on the same lattice */
    const long nr = gather_box(ce, &L, R_lo, R_hi, bufc);
    const double var_prev = var_of(bufc, nr);
    int mid[3];
    for (int a = 0; a < 3; ++a) mid[a] = R_lo[a] + (R_hi[a] - R_lo[a]) / 2;
    int best = -1, nvalid = 0;
    double best_m = 0.0, second_m = 0.0;
    int clo[8][3], chi[8][3], valid[8] = {0};
    double metric[8] = {0};
    for (int c = 0; c < nchild; ++c) {
      int ok = 1;
      for (int a = 0; a < 3; ++a) {
        if (a < g->dim) {
          int bit = (c >> a) & 1;
          clo[c][a] = bit ? mid[a] : R_lo[a];
          chi[c][a] = bit ? R_hi[a] : mid[a];
          if (chi[c][a] - clo[c][a] < r->min_segment) ok = 0;
        } else {
          clo[c][a] = R_lo[a];
          chi[c][a] = R_hi[a];
        }
      }
      if (!ok) continue;
      long nc = gather_box(ce, &L, clo[c], chi[c], bufc);
      if (nc == 0) continue;
      double mu = mean_of(bufc, nc), var = var_of(bufc, nc);
      double m;
      if (r->metric == ORC_METRIC_MEAN)
        m = mu;
      else if (r->metric == ORC_METRIC_VARIANCE)
        m = var;
      else if (r->metric == ORC_METRIC_HYBRID_UNCLIPPED)
        m = orc_hybrid_metric_unclipped(mu, var, var_prev);
      else
        m = orc_hybrid_metric(mu, var, var_prev);
      valid[c] = 1;
      metric[c] = m;
      if (nvalid == 0 || m > best_m) {
        if (nvalid > 0) second_m = best_m;
        best_m = m;
        best = c;
      } else if (nvalid == 1 || m > second_m) {
        second_m = m;
      }
      ++nvalid;
    }
    if (nvalid == 0) {
      res->stop_reason = ORC_STOP_MINSIZE;
      res->iters = i - 1;
      break;
    }
    const int take = path_take_child(path, li, nchild, best, best_m, valid, metric);
    if (take < 0) {
      st = ORC_ERR_ARG;
      break;
    }
    const int* best_lo = clo[take];
    const int* best_hi = chi[take];
    res->child[li] = take;
    res->n_children[li] = nvalid;
    res->metric_top[li] = metric[take];
    res->metric_gap[li] = nvalid > 1 ? rel_gap(best_m, second_m) : 1e300;
    int N_lo[3], N_hi[3];
    for (int a = 0; a < 3; ++a) {
      if (a < g->dim) {
        int side = best_hi[a] - best_lo[a];
        int grow = (side * r->frame_num + r->frame_den - 1) / r->frame_den;
        N_lo[a] = best_lo[a] - grow < 0 ? 0 : best_lo[a] - grow;
        N_hi[a] = best_hi[a] + grow > g->n[a] ? g->n[a] : best_hi[a] + grow;
      } else {
        N_lo[a] = best_lo[a];
        N_hi[a] = best_hi[a];
      }
      res->box_lo[li][a] = N_lo[a];
      res->box_hi[li][a] = N_hi[a];
    }
    /* Eq. 6-7 on the decimated profile, as in the paper's loop */
    long nb = gather_box(prof, &L0, N_lo, N_hi, bufb);
    double Wi, Bi;
    orc_scatter(bufa, (int)na, bufb, (int)nb, &Wi, &Bi);
    res->within[li] = Wi;
    res->between[li] = Bi;
    res->n_logged = i;
    if (i >= 2) {
      double mB = rel_gap(Bi, B_prev);
      double mW = rel_gap(W_prev, Wi);
      int cont = (Bi > B_prev) && (Wi < W_prev);
      res->stop_margin[li] = cont ? (mB < mW ? mB : mW) : (-mB > -mW ? -mB : -mW);
      if (!path_take_cont(path, li, cont)) {
        res->stop_reason = ORC_STOP_METRIC;
        res->iters = i - 1;
        break;
      }
    } else {
      res->stop_margin[li] = 1e300;
    }
    memcpy(R_lo, N_lo, sizeof N_lo);
    memcpy(R_hi, N_hi, sizeof N_hi);
    memcpy(bufa, bufb, sizeof(double) * (size_t)nb);
    na = nb;
    B_prev = Bi;
    W_prev = Wi;
    res->iters = i;
    if (i == max_iters) {
      res->stop_reason = ORC_STOP_CAP;
      break;
    }
  }
  free(prof); free(e); free(bufa); free(bufb); free(bufc);
  if (st != ORC_OK) {
    res->status = st;
    return st;
  }
  for (int a = 0; a < 3; ++a) {
    res->roi_lo[a] = R_lo[a];
    res->roi_hi[a] = R_hi[a];
  }
  /* final imaging of the region at full resolution, then its argmax */
  int step1[3] = {1, 1, 1}, cnt[3];
  for (int a = 0; a < 3; ++a) cnt[a] = R_hi[a] - R_lo[a];
  const long long nf = (long long)cnt[0] * cnt[1] * cnt[2];
  double* img = (double*)malloc(sizeof(double) * (size_t)(nf > 0 ? nf : 1));
  if (!img) {
    res->status = ORC_ERR_ARG;
    return ORC_ERR_ARG;
  }
  st = scan_image(&d, g, R_lo, step1, cnt, img);
  if (st != ORC_OK) {
    free(img);
    res->status = st;
    return st;
  }
  res->points_evaluated += nf;
  long long bestp = -1;
  for (long long p = 0; p < nf; ++p)
    if (bestp < 0 || img[p] > img[bestp]) bestp = p;
  if (bestp >= 0) {
    long long k[3] = {bestp % cnt[0], (bestp / cnt[0]) % cnt[1],
                      bestp / ((long long)cnt[0] * cnt[1])};
    for (int a = 0; a < 3; ++a) {
      res->loc_idx[a] = R_lo[a] + (int)k[a];
      res->loc_xyz[a] = g->origin[a] + (double)res->loc_idx[a] * g->pitch[a];
    }
    res->peak = img[bestp];
  }
  free(img);
  return ORC_OK;
}

int orc_presence(const float* traces, int M, int N, const float* antennas, const orc_grid* g,
                 double v, double fs, int window, int beamformer, const orc_rule* r,
                 int decimation2, orc_result* res1, orc_result* res2) {
  if (decimation2 < 1) return ORC_ERR_ARG;
  int st = orc_localize(traces, M, N, antennas, g, v, fs, window, beamformer, r, res1);
  if (st != ORC_OK) return st;
  orc_rule r2 = *r;
  r2.mode = ORC_DECIM_MANUAL;
  r2.decimation = decimation2;
  st = orc_localize(traces, M, N, antennas, g, v, fs, window, beamformer, &r2, res2);
  if (st != ORC_OK) return st;
  if (res1->loc_idx[0] < 0 || res2->loc_idx[0] < 0) return 0; /* nothing located */
  for (int a = 0; a < 3; ++a)
    if (res1->loc_idx[a] != res2->loc_idx[a]) return 0;
  return 1;
}
