/*
 * cox_oracle.c -- plain FP64 CPU oracle for the regularized stratified / time-varying Cox
 * model fitted by cyclic coordinate descent (Yang, Schuemie & Suchard, arXiv 2310.16238).
 *
 * TEST INFRASTRUCTURE ONLY. This is the slow, obviously-correct reference that the CUDA
 * library is checked against. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it; the product path never does. It shares no code, header,
 * table or helper with the CUDA library.
 *
 * What it follows (paper sections and equations):
 *   - stratified partial likelihood, eq. (strat_l), §2.1, with Breslow risk sets
 *     R_k(Y) = {r : Y_kr >= Y} inside the stratum;
 *   - time-varying covariates as counting-process rows (start, stop], §2.2 eq. (time_cov_l):
 *     a row is at risk at t iff start < t <= stop;
 *   - the gradient and Hessian of the negative log partial likelihood, eqs. (strat_g) and
 *     (strat_h), §2.4, evaluated through segmented scans of D = exp(X beta), N1 = X_j * D,
 *     N2 = X_j * X_j * D over the time-ordered, stratum-concatenated rows, §2.6-§2.7,
 *     eqs. (parallel_g), (parallel_h), (parallel_d), (parallel_n1), (parallel_n2);
 *   - the incremental linear predictor update, eq. (parallel_xb);
 *   - cyclic coordinate descent with the 1-D Newton step, eq. (newton), the trust region
 *     and the L1 directional-derivative rule of §2.4.
 *
 * Readings where the paper is silent or ambiguous:
 *   R1 ties: every event at time t in stratum k sees the whole risk set {r : Y_r >= t}
 *      (Breslow); with rows in decreasing time order the scan is read at the LAST row of
 *      the tie block, i.e. the first row of the block in increasing order.
 *   R2 trust region: Delta_j starts at 1; the Newton step is clipped to [-Delta_j, Delta_j];
 *      after every visit Delta_j <- max(2 |applied step|, Delta_j / 2).
 *   R3 L1 away from 0: step on g' + gamma sgn(beta_j); a step that would cross zero stops at 0.
 *   R4 L2: penalty sum_j m_j beta_j^2 / (2 sigma^2) (Gaussian prior variance sigma^2).
 *   R5 convergence: after each full sweep, |obj_new - obj_old| <= tol * |obj_new| on the
 *      penalized objective obj = -loglik + penalty; at most max_sweeps sweeps.
 *   R6 g'' <= 0 (after the penalty) or not finite: the coordinate is skipped (step 0).
 *   R7 start-stop risk sets are formed by an entry/exit sweep over time (a row enters the
 *      running sums when t falls to its stop and leaves when t falls to its start).
 *
 * All sums over many terms use Neumaier's compensated summation (A. Neumaier, 1974,
 * "Rundungsfehleranalyse einiger Verfahren zur Summation endlicher Summen").
 * Build: cc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so x86 and Arm agree).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OCX_OK 0
#define OCX_E_INVALID (-1)
#define OCX_E_UNSORTED (-2)
#define OCX_E_OOM (-3)

#define OCX_PEN_NONE 0
#define OCX_PEN_L1 1
#define OCX_PEN_L2 2

typedef struct {
  int64_t n;              /* rows */
  int32_t p;              /* columns */
  const int32_t *stop;    /* [n] integer times, sorted ascending within stratum */
  const int32_t *start;   /* [n] or NULL: counting-process entry times, start < stop */
  const uint8_t *event;   /* [n] 0/1 */
  const int32_t *stratum; /* [n] or NULL (one stratum); primary sort key */
  const int64_t *col_ptr; /* [p+1] CSC */
  const int32_t *row_idx; /* [nnz] ascending within a column */
  const double *val;      /* [nnz] or NULL (binary X) */
} ocx_data;

typedef struct {
  int32_t penalty;          /* OCX_PEN_* */
  double lambda;            /* L1 gamma */
  double l2_var;            /* L2 prior variance sigma^2 */
  const uint8_t *penalize;  /* [p] or NULL (all penalized) */
  double tol;
  int32_t max_sweeps;
} ocx_options;

typedef struct {
  int32_t sweeps;
  int64_t coord_updates;
  double loglik;
  double objective;
  int32_t converged;
} ocx_info;

/* ---------------------------------------------------------------- compensated sums */
typedef struct { double s, c; } ksum;

static void kadd(ksum *a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}
static double kval(const ksum *a) { return a->s + a->c; }

/* ---------------------------------------------------------------- helpers */
static int32_t stratum_of(const ocx_data *d, int64_t r) { return d->stratum ? d->stratum[r] : 0; }

/* Paper §2.6: segmented inclusive scan with the flag-value operator
 *   (f_i, a_i) (+)s (f_j, a_j) = (f_i | f_j, f_j ? a_j : a_i + a_j),
 * applied left to right. Plain (uncompensated) so that it is the operator as written. */
void ocx_segscan(int64_t n, const double *a, const uint8_t *f, double *b) {
  double acc = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    acc = (i == 0 || f[i]) ? a[i] : acc + a[i];
    b[i] = acc;
  }
}

/* The same operator with a compensated accumulator (used by the likelihood code). */
static void segscan_comp(int64_t n, const double *a, const uint8_t *f, double *b) {
  ksum acc = {0.0, 0.0};
  for (int64_t i = 0; i < n; ++i) {
    if (i == 0 || f[i]) { acc.s = a[i]; acc.c = 0.0; }
    else kadd(&acc, a[i]);
    b[i] = kval(&acc);
  }
}

/* ---------------------------------------------------------------- validation */
int ocx_validate(const ocx_data *d) {
  if (d->n < 0 || d->p < 0 || !d->stop || !d->event || !d->col_ptr) return OCX_E_INVALID;
  for (int64_t r = 0; r < d->n; ++r) {
    if (d->event[r] > 1) return OCX_E_INVALID;
    if (d->start && !(d->start[r] < d->stop[r])) return OCX_E_INVALID;
    if (r > 0) {
      int32_t k0 = stratum_of(d, r - 1), k1 = stratum_of(d, r);
      if (k1 < k0 || (k1 == k0 && d->stop[r] < d->stop[r - 1])) return OCX_E_UNSORTED;
    }
  }
  if (d->col_ptr[0] != 0) return OCX_E_INVALID;
  for (int32_t j = 0; j < d->p; ++j) {
    if (d->col_ptr[j + 1] < d->col_ptr[j]) return OCX_E_INVALID;
    for (int64_t q = d->col_ptr[j]; q < d->col_ptr[j + 1]; ++q) {
      if (d->row_idx[q] < 0 || d->row_idx[q] >= d->n) return OCX_E_INVALID;
      if (q > d->col_ptr[j] && d->row_idx[q] <= d->row_idx[q - 1]) return OCX_E_INVALID;
    }
  }
  return OCX_OK;
}

/* ---------------------------------------------------------------- integer metadata */
/* Stratum offsets: seg_off[k] = first row of the k-th stratum, seg_off[K] = n. Returns K. */
int64_t ocx_strata(const ocx_data *d, int64_t *seg_off) {
  int64_t K = 0;
  for (int64_t r = 0; r < d->n; ++r)
    if (r == 0 || stratum_of(d, r) != stratum_of(d, r - 1)) seg_off[K++] = r;
  seg_off[K] = d->n;
  return K;
}

/* Tie groups (paper eq. strat_l with R1): one group per (stratum, time) that has >= 1 event.
 * head[g] = first row (increasing order) with that (stratum, stop); d[g] = number of events;
 * t[g] = the time; k[g] = the stratum id. Returns G. Arrays must hold n entries. */
int64_t ocx_tie_groups(const ocx_data *d, int64_t *head, int32_t *dcount, int32_t *t, int32_t *k) {
  int64_t G = 0;
  int64_t r = 0;
  while (r < d->n) {
    int64_t e = r;
    int32_t cnt = 0;
    while (e < d->n && stratum_of(d, e) == stratum_of(d, r) && d->stop[e] == d->stop[r]) {
      cnt += d->event[e];
      ++e;
    }
    if (cnt > 0) {
      head[G] = r; dcount[G] = cnt; t[G] = d->stop[r]; k[G] = stratum_of(d, r);
      ++G;
    }
    r = e;
  }
  return G;
}

/* Number of rows at risk at each tie group, straight from the definition of the risk set
 * (stop >= t, and start < t for counting-process rows), inside the group's stratum. */
void ocx_risk_count(const ocx_data *d, int64_t G, const int32_t *t, const int32_t *k, int64_t *count) {
  for (int64_t g = 0; g < G; ++g) {
    int64_t c = 0;
    for (int64_t r = 0; r < d->n; ++r) {
      if (stratum_of(d, r) != k[g]) continue;
      if (d->stop[r] >= t[g] && (!d->start || d->start[r] < t[g])) ++c;
    }
    count[g] = c;
  }
}

/* delta' X_j for every column (paper §2.7, the first term of eq. parallel_g). */
void ocx_dX(const ocx_data *d, double *dX) {
  for (int32_t j = 0; j < d->p; ++j) {
    ksum s = {0.0, 0.0};
    for (int64_t q = d->col_ptr[j]; q < d->col_ptr[j + 1]; ++q)
      if (d->event[d->row_idx[q]]) kadd(&s, d->val ? d->val[q] : 1.0);
    dX[j] = kval(&s);
  }
}

/* Linear predictor eta = X beta, accumulated column by column (j = 0..p-1). */
void ocx_eta(const ocx_data *d, const double *beta, double *eta) {
  for (int64_t r = 0; r < d->n; ++r) eta[r] = 0.0;
  for (int32_t j = 0; j < d->p; ++j) {
    if (beta[j] == 0.0) continue;
    for (int64_t q = d->col_ptr[j]; q < d->col_ptr[j + 1]; ++q) {
      double x = d->val ? d->val[q] : 1.0;
      eta[d->row_idx[q]] = eta[d->row_idx[q]] + x * beta[j];
    }
  }
}

/* ---------------------------------------------------------------- fit context */
typedef struct {
  const ocx_data *d;
  int64_t G;
  int64_t *head;
  int32_t *dcount, *t, *k;
  int64_t *group_of_row;  /* tie group of each event row, -1 otherwise */
  uint8_t *flag_desc;     /* head flags in decreasing-time order (§2.7) */
  int64_t *sidx;          /* rows ordered by (stratum, start) for counting-process data */
  int64_t *seg_off;
  int64_t K;
  double *xj;             /* dense column scratch [n] */
  double *bufA, *bufB, *bufC, *scanA, *scanB, *scanC; /* [n] */
} ctx_t;

/* qsort has no context argument in C99; the oracle is single-threaded, so a file-scope
 * pointer carries the data to the comparator. */
static const ocx_data *cmp_d;
static int cmp_start(const void *a, const void *b) {
  int64_t ra = *(const int64_t *)a, rb = *(const int64_t *)b;
  int32_t ka = stratum_of(cmp_d, ra), kb = stratum_of(cmp_d, rb);
  if (ka != kb) return ka < kb ? -1 : 1;
  if (cmp_d->start[ra] != cmp_d->start[rb]) return cmp_d->start[ra] < cmp_d->start[rb] ? -1 : 1;
  return ra < rb ? -1 : (ra > rb ? 1 : 0);
}

static void ctx_free(ctx_t *c) {
  free(c->head); free(c->dcount); free(c->t); free(c->k); free(c->group_of_row);
  free(c->flag_desc); free(c->sidx); free(c->seg_off); free(c->xj);
  free(c->bufA); free(c->bufB); free(c->bufC); free(c->scanA); free(c->scanB); free(c->scanC);
  memset(c, 0, sizeof(*c));
}

static int ctx_init(ctx_t *c, const ocx_data *d) {
  memset(c, 0, sizeof(*c));
  c->d = d;
  int64_t n = d->n > 0 ? d->n : 1;
  c->head = malloc(sizeof(int64_t) * n); c->dcount = malloc(sizeof(int32_t) * n);
  c->t = malloc(sizeof(int32_t) * n); c->k = malloc(sizeof(int32_t) * n);
  c->group_of_row = malloc(sizeof(int64_t) * n); c->flag_desc = malloc(n);
  c->seg_off = malloc(sizeof(int64_t) * (n + 1)); c->xj = calloc(n, sizeof(double));
  c->bufA = malloc(sizeof(double) * n); c->bufB = malloc(sizeof(double) * n);
  c->bufC = malloc(sizeof(double) * n); c->scanA = malloc(sizeof(double) * n);
  c->scanB = malloc(sizeof(double) * n); c->scanC = malloc(sizeof(double) * n);
  if (!c->head || !c->dcount || !c->t || !c->k || !c->group_of_row || !c->flag_desc || !c->seg_off ||
      !c->xj || !c->bufA || !c->bufB || !c->bufC || !c->scanA || !c->scanB || !c->scanC) {
    ctx_free(c);
    return OCX_E_OOM;
  }
  c->G = ocx_tie_groups(d, c->head, c->dcount, c->t, c->k);
  c->K = ocx_strata(d, c->seg_off);
  for (int64_t r = 0; r < d->n; ++r) c->group_of_row[r] = -1;
  for (int64_t g = 0; g < c->G; ++g)
    for (int64_t r = c->head[g]; r < d->n && stratum_of(d, r) == c->k[g] && d->stop[r] == c->t[g]; ++r)
      if (d->event[r]) c->group_of_row[r] = g;
  /* decreasing-time order: position q holds row n-1-q; a segment starts at the first
   * position of each stratum in that order, i.e. at the last row of the stratum */
  for (int64_t q = 0; q < d->n; ++q) {
    int64_t r = d->n - 1 - q;
    c->flag_desc[q] = (q == 0 || stratum_of(d, r) != stratum_of(d, r + 1)) ? 1 : 0;
  }
  if (d->start) {
    c->sidx = malloc(sizeof(int64_t) * n);
    if (!c->sidx) { ctx_free(c); return OCX_E_OOM; }
    for (int64_t r = 0; r < d->n; ++r) c->sidx[r] = r;
    cmp_d = d;
    qsort(c->sidx, (size_t)d->n, sizeof(int64_t), cmp_start);
  }
  return OCX_OK;
}

/* Risk-set sums at every tie group for column j, given D = exp(eta) per row:
 *   S0_g = sum_{r in R(t_g)} D_r,  S1_g = sum x_rj D_r,  S2_g = sum x_rj^2 D_r.
 * Right-censored data: segmented scans in decreasing-time order (§2.7). Counting-process
 * data: entry/exit sweep (reading R7). */
static void risk_sums(ctx_t *c, const double *D, int32_t j, double *S0, double *S1, double *S2) {
  const ocx_data *d = c->d;
  int64_t n = d->n;
  /* dense X_j (paper: X_j is an N-vector; zeros where the CSC has no entry) */
  if (j >= 0)
    for (int64_t q = d->col_ptr[j]; q < d->col_ptr[j + 1]; ++q) c->xj[d->row_idx[q]] = d->val ? d->val[q] : 1.0;
  if (!d->start) {
    for (int64_t q = 0; q < n; ++q) {
      int64_t r = n - 1 - q;
      double x = j >= 0 ? c->xj[r] : 0.0;
      c->bufA[q] = D[r];            /* eq. parallel_d  */
      c->bufB[q] = x * D[r];        /* eq. parallel_n1 */
      c->bufC[q] = x * x * D[r];    /* eq. parallel_n2 */
    }
    segscan_comp(n, c->bufA, c->flag_desc, c->scanA);
    segscan_comp(n, c->bufB, c->flag_desc, c->scanB);
    segscan_comp(n, c->bufC, c->flag_desc, c->scanC);
    for (int64_t g = 0; g < c->G; ++g) {
      int64_t q = n - 1 - c->head[g];   /* reading R1 */
      S0[g] = c->scanA[q]; S1[g] = c->scanB[q]; S2[g] = c->scanC[q];
    }
  } else {
    /* per stratum, tie groups by decreasing time; rows enter when t <= stop, leave when t <= start */
    int64_t g = c->G - 1;
    for (int64_t kk = c->K - 1; kk >= 0; --kk) {
      int64_t a = c->seg_off[kk], b = c->seg_off[kk + 1];
      int64_t ps = b - 1, pq = b - 1;   /* stop order and start order (sidx) share stratum bounds */
      ksum s0 = {0, 0}, s1 = {0, 0}, s2 = {0, 0};
      int32_t kid = stratum_of(d, a);
      for (; g >= 0 && c->k[g] == kid; --g) {
        int32_t tg = c->t[g];
        while (ps >= a && d->stop[ps] >= tg) {
          double x = j >= 0 ? c->xj[ps] : 0.0;
          kadd(&s0, D[ps]); kadd(&s1, x * D[ps]); kadd(&s2, x * x * D[ps]);
          --ps;
        }
        while (pq >= a && d->start[c->sidx[pq]] >= tg) {
          int64_t r = c->sidx[pq];
          double x = j >= 0 ? c->xj[r] : 0.0;
          kadd(&s0, -D[r]); kadd(&s1, -(x * D[r])); kadd(&s2, -(x * x * D[r]));
          --pq;
        }
        S0[g] = kval(&s0); S1[g] = kval(&s1); S2[g] = kval(&s2);
      }
    }
  }
  if (j >= 0)
    for (int64_t q = d->col_ptr[j]; q < d->col_ptr[j + 1]; ++q) c->xj[d->row_idx[q]] = 0.0;
}

/* g'(beta_j), g''(beta_j) of the negative log partial likelihood, eqs. strat_g / strat_h:
 * a sum over event rows i of the risk-set ratios at Y_i. */
static void grad_hess_from_sums(ctx_t *c, const double *S0, const double *S1, const double *S2,
                                double dXj, double *g1, double *g2) {
  const ocx_data *d = c->d;
  ksum a = {0, 0}, b = {0, 0};
  kadd(&a, -dXj);
  for (int64_t r = 0; r < d->n; ++r) {
    int64_t g = c->group_of_row[r];
    if (g < 0) continue;                 /* delta_i = 0 */
    double q1 = S1[g] / S0[g];
    kadd(&a, q1);
    kadd(&b, S2[g] / S0[g]);
    kadd(&b, -(q1 * q1));
  }
  *g1 = kval(&a);
  *g2 = kval(&b);
}

/* log partial likelihood, eq. strat_l: sum over event rows of eta_i - log S0(Y_i). */
static double loglik_from_sums(ctx_t *c, const double *eta, const double *S0) {
  const ocx_data *d = c->d;
  ksum a = {0, 0};
  for (int64_t r = 0; r < d->n; ++r) {
    int64_t g = c->group_of_row[r];
    if (g < 0) continue;
    kadd(&a, eta[r]);
    kadd(&a, -log(S0[g]));
  }
  return kval(&a);
}

/* ---------------------------------------------------------------- public evaluations */
int64_t ocx_num_groups(const ocx_data *d) {
  int64_t G = 0, r = 0;
  while (r < d->n) {
    int64_t e = r; int32_t cnt = 0;
    while (e < d->n && stratum_of(d, e) == stratum_of(d, r) && d->stop[e] == d->stop[r]) { cnt += d->event[e]; ++e; }
    if (cnt > 0) ++G;
    r = e;
  }
  return G;
}

/* Risk-set sums at every tie group for column j (j < 0: S1 = S2 = 0), at linear predictor eta. */
int ocx_risk_sums(const ocx_data *d, const double *eta, int32_t j, double *S0, double *S1, double *S2) {
  ctx_t c;
  int rc = ctx_init(&c, d);
  if (rc) return rc;
  double *D = malloc(sizeof(double) * (d->n > 0 ? d->n : 1));
  if (!D) { ctx_free(&c); return OCX_E_OOM; }
  for (int64_t r = 0; r < d->n; ++r) D[r] = exp(eta[r]);
  risk_sums(&c, D, j, S0, S1, S2);
  free(D);
  ctx_free(&c);
  return OCX_OK;
}

/* Unpenalized g'(beta_j), g''(beta_j) of -loglik at eta, for the listed coordinates. */
int ocx_grad_hess(const ocx_data *d, const double *eta, int32_t ncols, const int32_t *cols, double *g1, double *g2) {
  ctx_t c;
  int rc = ctx_init(&c, d);
  if (rc) return rc;
  int64_t G = c.G > 0 ? c.G : 1;
  double *D = malloc(sizeof(double) * (d->n > 0 ? d->n : 1));
  double *S0 = malloc(sizeof(double) * G), *S1 = malloc(sizeof(double) * G), *S2 = malloc(sizeof(double) * G);
  double *dX = malloc(sizeof(double) * (d->p > 0 ? d->p : 1));
  if (!D || !S0 || !S1 || !S2 || !dX) { free(D); free(S0); free(S1); free(S2); free(dX); ctx_free(&c); return OCX_E_OOM; }
  for (int64_t r = 0; r < d->n; ++r) D[r] = exp(eta[r]);
  ocx_dX(d, dX);
  for (int32_t i = 0; i < ncols; ++i) {
    int32_t j = cols[i];
    risk_sums(&c, D, j, S0, S1, S2);
    grad_hess_from_sums(&c, S0, S1, S2, dX[j], &g1[i], &g2[i]);
  }
  free(D); free(S0); free(S1); free(S2); free(dX);
  ctx_free(&c);
  return OCX_OK;
}

/* log partial likelihood at eta (unpenalized). */
int ocx_loglik(const ocx_data *d, const double *eta, double *out) {
  ctx_t c;
  int rc = ctx_init(&c, d);
  if (rc) return rc;
  int64_t G = c.G > 0 ? c.G : 1;
  double *D = malloc(sizeof(double) * (d->n > 0 ? d->n : 1));
  double *S0 = malloc(sizeof(double) * G), *S1 = malloc(sizeof(double) * G), *S2 = malloc(sizeof(double) * G);
  if (!D || !S0 || !S1 || !S2) { free(D); free(S0); free(S1); free(S2); ctx_free(&c); return OCX_E_OOM; }
  for (int64_t r = 0; r < d->n; ++r) D[r] = exp(eta[r]);
  risk_sums(&c, D, -1, S0, S1, S2);
  *out = loglik_from_sums(&c, eta, S0);
  free(D); free(S0); free(S1); free(S2);
  ctx_free(&c);
  return OCX_OK;
}

/* ---------------------------------------------------------------- the coordinate step */
/* One CCD step for coordinate j (§2.4): penalty, Newton step eq. (newton), trust region,
 * L1 directional derivatives at the origin, and the trust-region update (readings R2-R4, R6).
 * g1, g2 are the unpenalized derivatives of -loglik. Returns the applied step; *tr is updated. */
double ocx_step(double g1, double g2, double beta_j, double *tr, int32_t penalty, double lambda,
                double l2_var, int32_t penalized) {
  double gamma = 0.0;
  if (penalized && penalty == OCX_PEN_L2) {
    g1 = g1 + beta_j / l2_var;
    g2 = g2 + 1.0 / l2_var;
  }
  if (penalized && penalty == OCX_PEN_L1) gamma = lambda;
  double step;
  if (!(g2 > 0.0) || !isfinite(g1) || !isfinite(g2)) {
    step = 0.0;
  } else if (gamma > 0.0) {
    if (beta_j == 0.0) {
      if (g1 + gamma < 0.0) step = -(g1 + gamma) / g2;        /* descent in the + direction */
      else if (g1 - gamma > 0.0) step = -(g1 - gamma) / g2;   /* descent in the - direction */
      else step = 0.0;                                        /* both directional derivatives >= 0 */
    } else {
      step = -(g1 + (beta_j > 0.0 ? gamma : -gamma)) / g2;
    }
  } else {
    step = -g1 / g2;
  }
  if (fabs(step) > *tr) step = step > 0.0 ? *tr : -*tr;
  if (gamma > 0.0 && beta_j != 0.0) {
    double nb = beta_j + step;
    if ((beta_j > 0.0 && nb < 0.0) || (beta_j < 0.0 && nb > 0.0)) step = -beta_j;
  }
  double t2 = 2.0 * fabs(step), th = 0.5 * *tr;
  *tr = t2 > th ? t2 : th;
  return step;
}

static double penalty_value(const ocx_options *o, int32_t p, const double *beta) {
  ksum s = {0, 0};
  for (int32_t j = 0; j < p; ++j) {
    if (o->penalize && !o->penalize[j]) continue;
    if (o->penalty == OCX_PEN_L1) kadd(&s, o->lambda * fabs(beta[j]));
    else if (o->penalty == OCX_PEN_L2) kadd(&s, beta[j] * beta[j] / (2.0 * o->l2_var));
  }
  return kval(&s);
}

/* Cyclic coordinate descent (§2.4), starting from beta0 (NULL = 0), coordinates j = 0..p-1
 * in order each sweep. eta and D are maintained incrementally at the nonzeros of X_j
 * (eq. parallel_xb). Convergence per reading R5. Returns 0, or 1 when not converged. */
int ocx_fit(const ocx_data *d, const ocx_options *o, const double *beta0, double *beta, ocx_info *info) {
  ctx_t c;
  int rc = ctx_init(&c, d);
  if (rc) return rc;
  int64_t n = d->n > 0 ? d->n : 1, G = c.G > 0 ? c.G : 1;
  int32_t p = d->p;
  double *eta = malloc(sizeof(double) * n), *D = malloc(sizeof(double) * n);
  double *S0 = malloc(sizeof(double) * G), *S1 = malloc(sizeof(double) * G), *S2 = malloc(sizeof(double) * G);
  double *dX = malloc(sizeof(double) * (p > 0 ? p : 1)), *tr = malloc(sizeof(double) * (p > 0 ? p : 1));
  if (!eta || !D || !S0 || !S1 || !S2 || !dX || !tr) {
    free(eta); free(D); free(S0); free(S1); free(S2); free(dX); free(tr); ctx_free(&c);
    return OCX_E_OOM;
  }
  for (int32_t j = 0; j < p; ++j) { beta[j] = beta0 ? beta0[j] : 0.0; tr[j] = 1.0; }
  ocx_eta(d, beta, eta);
  for (int64_t r = 0; r < d->n; ++r) D[r] = exp(eta[r]);
  ocx_dX(d, dX);

  risk_sums(&c, D, -1, S0, S1, S2);
  double ll = loglik_from_sums(&c, eta, S0);
  double obj_prev = -ll + penalty_value(o, p, beta), obj = obj_prev;
  int32_t sweeps = 0, converged = 0;
  while (sweeps < o->max_sweeps) {
    for (int32_t j = 0; j < p; ++j) {
      double g1, g2;
      risk_sums(&c, D, j, S0, S1, S2);
      grad_hess_from_sums(&c, S0, S1, S2, dX[j], &g1, &g2);
      int32_t pen = o->penalize ? o->penalize[j] : 1;
      double step = ocx_step(g1, g2, beta[j], &tr[j], o->penalty, o->lambda, o->l2_var, pen);
      if (step != 0.0) {
        beta[j] = beta[j] + step;
        for (int64_t q = d->col_ptr[j]; q < d->col_ptr[j + 1]; ++q) {
          int64_t r = d->row_idx[q];
          double x = d->val ? d->val[q] : 1.0;
          eta[r] = eta[r] + x * step;   /* eq. parallel_xb */
          D[r] = exp(eta[r]);           /* eq. parallel_d at the touched rows */
        }
      }
    }
    ++sweeps;
    risk_sums(&c, D, -1, S0, S1, S2);
    ll = loglik_from_sums(&c, eta, S0);
    obj = -ll + penalty_value(o, p, beta);
    if (fabs(obj - obj_prev) <= o->tol * fabs(obj)) { converged = 1; break; }
    obj_prev = obj;
  }
  if (info) {
    info->sweeps = sweeps;
    info->coord_updates = (int64_t)sweeps * p;
    info->loglik = ll;
    info->objective = obj;
    info->converged = converged;
  }
  free(eta); free(D); free(S0); free(S1); free(S2); free(dX); free(tr);
  ctx_free(&c);
  return converged ? OCX_OK : 1;
}

/* A bounded sample of the fit's work, for timing: `ncoords` coordinate evaluations
 * (risk sums + gradient/Hessian + step + eta update) starting from beta = 0. */
int ocx_time_sample(const ocx_data *d, const ocx_options *o, int32_t ncoords, double *checksum, double *beta_out) {
  ctx_t c;
  int rc = ctx_init(&c, d);
  if (rc) return rc;
  int64_t n = d->n > 0 ? d->n : 1, G = c.G > 0 ? c.G : 1;
  int32_t p = d->p;
  double *eta = calloc(n, sizeof(double)), *D = malloc(sizeof(double) * n);
  double *S0 = malloc(sizeof(double) * G), *S1 = malloc(sizeof(double) * G), *S2 = malloc(sizeof(double) * G);
  double *dX = malloc(sizeof(double) * (p > 0 ? p : 1)), *tr = malloc(sizeof(double) * (p > 0 ? p : 1));
  double *beta = calloc(p > 0 ? p : 1, sizeof(double));
  if (!eta || !D || !S0 || !S1 || !S2 || !dX || !tr || !beta) {
    free(eta); free(D); free(S0); free(S1); free(S2); free(dX); free(tr); free(beta); ctx_free(&c);
    return OCX_E_OOM;
  }
  for (int64_t r = 0; r < d->n; ++r) D[r] = 1.0;
  for (int32_t j = 0; j < p; ++j) tr[j] = 1.0;
  ocx_dX(d, dX);
  double acc = 0.0;
  for (int32_t i = 0; i < ncoords && p > 0; ++i) {
    int32_t j = i % p;
    double g1, g2;
    risk_sums(&c, D, j, S0, S1, S2);
    grad_hess_from_sums(&c, S0, S1, S2, dX[j], &g1, &g2);
    double step = ocx_step(g1, g2, beta[j], &tr[j], o->penalty, o->lambda, o->l2_var, o->penalize ? o->penalize[j] : 1);
    if (step != 0.0) {
      beta[j] += step;
      for (int64_t q = d->col_ptr[j]; q < d->col_ptr[j + 1]; ++q) {
        int64_t r = d->row_idx[q];
        eta[r] = eta[r] + (d->val ? d->val[q] : 1.0) * step;
        D[r] = exp(eta[r]);
      }
    }
    acc += g1 + g2;
  }
  *checksum = acc;
  if (beta_out)
    for (int32_t j = 0; j < p; ++j) beta_out[j] = beta[j];
  free(eta); free(D); free(S0); free(S1); free(S2); free(dX); free(tr); free(beta);
  ctx_free(&c);
  return OCX_OK;
}
