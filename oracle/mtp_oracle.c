/*
 * mtp_oracle.c -- plain, slow FP64 CPU oracle for one Model Tensor Planning
 * (MTP) planner iteration (arXiv 2505.01059, Alg. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no source, header, table or
 * constant generator with the CUDA path: the counter-based generator (Philox4x32-10,
 * Salmon et al., SC'11) and every step of the method are written here a second
 * time, from the paper and the published generator definition.
 *
 * Every function follows the paper's steps in its order and notation; there is
 * no blocking, fusion or reordering.  Equation numbers count the paper's
 * labelled equations: Eq. 1 total variation, Eq. 2 cumulative cost, Eq. 3
 * B-spline, Eq. 4 Cox-de Boor recursion, Eq. 5 Akima polynomial, Eq. 6 Akima
 * slope, Eq. 7 Akima coefficients.  The unlabelled CEM moment update of
 * Sec. 2.1 is cited as "Sec. 2.1, CEM update".
 *
 * Where the paper is silent or garbled the oracle takes these readings:
 *   - Alg. 1 draws indices uniformly over the N nodes, 0-based here.
 *   - Alg. 2 samples the graph in control space (M x N x n), not state space.
 *   - P = min(floor(beta*B), B-1); B-P-1 local samples; the nominal mean is
 *     always the last candidate.
 *   - Def. 2 has M+p+1 uniform knots and therefore M basis functions, one per
 *     graph layer.  Evaluation times: "valid span" (default) maps j/(H-1) onto
 *     [t_p, t_M] where the basis sums to one; "paper literal" uses t_j = j/H.
 *   - Eq. 4's degree-0 indicator is half-open [t_i, t_{i+1}); at the right end
 *     of the valid span (t = t_M) the last interval is taken as closed.
 *   - Def. 3 knots: default t_i = i/(M-1) evaluated at j/(H-1); paper literal
 *     t_i = i/M evaluated at j/H (the last cubic extrapolates).
 *   - Eq. 6 with a zero denominator uses the mean of the two adjacent slopes.
 *   - Alg. 2's new spread is a standard deviation with floor sigma_m, and the
 *     softmax weights are taken after subtracting the best elite cost.
 *   - Controls are clamped to the box before the rollout.
 *   - Elite order is the total order on (cost, index); NaN costs count as +inf.
 *
 * Philox counter layout (shared convention, implemented independently on each
 * side): key = (seed low 32 bits, seed high 32 bits), counter =
 * (index, sub-index/4, iteration, stream tag); each call yields four words.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXN 32   /* maximum control dimension */
#define OR_MAXL 18   /* maximum number of links */
#define OR_MAXOBS 8  /* maximum number of obstacles */

enum { OR_DYN_POINTMASS = 0, OR_DYN_CHAIN = 1, OR_DYN_LEGGED = 2 };
enum { OR_INTERP_LINEAR = 0, OR_INTERP_BSPLINE = 1, OR_INTERP_AKIMA = 2 };
enum { OR_TIME_VALID_SPAN = 0, OR_TIME_PAPER_LITERAL = 1 };
enum { OR_UPDATE_SOFTMAX = 0, OR_UPDATE_PLAIN_CEM = 1 };
enum { OR_DR_NONE = 0, OR_DR_PER_SAMPLE = 1, OR_DR_SHARED = 2 };
enum { OR_TAG_GRAPH = 1, OR_TAG_PATH = 2, OR_TAG_LOCAL = 3, OR_TAG_PARAM_SAMPLE = 4,
       OR_TAG_PARAM_MODEL = 5 };

/* The oracle's own description of one planning problem. */
typedef struct {
  int32_t dyn, n, d, H;
  int32_t M, N, B, P, E;
  int32_t interp, degree, time_mapping, update_rule;
  int32_t dr_mode, R;
  uint64_t seed;
  double dt, lambda, alpha, sigma_min;
  double u_min[OR_MAXN], u_max[OR_MAXN];
  /* task: target (point-mass goal / chain reach target / legged: [0]=height, [1]=velocity) */
  double target[OR_MAXN];
  double w_target, w_obs, w_ctrl, w_term;
  int32_t n_obs;
  double obs_c[OR_MAXOBS][OR_MAXN];
  double obs_r[OR_MAXOBS];
  /* domain-randomisation scale range */
  double dr_lo, dr_hi;
  /* links (chain / legged) */
  int32_t n_links;
  double mass[OR_MAXL], length[OR_MAXL];
  double gravity;
  /* legged ground contact */
  double k_contact, c_contact, mu_friction, v_slip;
  double w_height, w_pitch, w_vel;
  /* precision of the B-spline contraction: 0 FP64; 1 operands (basis value
   * and knot, each first rounded to FP32) rounded to BF16, products and sums
   * exact here (the GPU sums in FP32) */
  int32_t bf16_basis;
} or_problem;

/* ------------------------------------------------------------------------- */
/* Counter-based generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
/* ------------------------------------------------------------------------- */

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint64_t MUL0 = 0xD2511F53u, MUL1 = 0xCD9E8D57u;
  const uint32_t WEYL0 = 0x9E3779B9u, WEYL1 = 0xBB67AE85u;
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = MUL0 * (uint64_t)c[0];
    uint64_t p1 = MUL1 * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    k0 += WEYL0; k1 += WEYL1;
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

static uint32_t draw_word(uint64_t seed, uint32_t a, uint32_t b, uint32_t iter, uint32_t tag) {
  /* word (b & 3) of the call at counter (a, b / 4, iter, tag) */
  uint32_t ctr[4] = {a, b >> 2, iter, tag};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t out[4];
  or_philox4x32_10(ctr, key, out);
  return out[b & 3u];
}

/* uniform in [0, 1): the top 24 bits of a word */
static double unit_uniform(uint32_t r) { return (double)(r >> 8) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------------- */
/* Def. 1 and Alg. 1: random multipartite graph and path sampling.            */
/* ------------------------------------------------------------------------- */

/* Number of graph samples P = floor(beta*B), capped at B-1 so the nominal mean
 * always has a slot (Alg. 2, local sampling needs B-P-1 >= 0). */
int32_t or_num_graph_samples(double beta, int32_t B) {
  int32_t P = (int32_t)floor(beta * (double)B);
  if (P > B - 1) P = B - 1;
  if (P < 0) P = 0;
  return P;
}

/* Def. 1: Z[m][j][i] uniform over the control box U, one layer per m. */
void or_graph_Z(const or_problem* pr, uint32_t iter, double* Z) {
  for (int m = 0; m < pr->M; ++m)
    for (int j = 0; j < pr->N; ++j)
      for (int i = 0; i < pr->n; ++i) {
        uint32_t r = draw_word(pr->seed, (uint32_t)(m * pr->N + j), (uint32_t)i, iter, OR_TAG_GRAPH);
        Z[((size_t)m * pr->N + j) * pr->n + i] =
            pr->u_min[i] + (pr->u_max[i] - pr->u_min[i]) * unit_uniform(r);
      }
}

/* Alg. 1, first step: I = randint((P, M), over the N nodes), with replacement.
 * The index is the high word of r*N, which is uniform over {0..N-1} up to
 * 2^-32 bias (Lemire's multiply-high mapping). */
void or_path_indices(const or_problem* pr, uint32_t iter, int32_t P, int32_t* I) {
  for (int b = 0; b < P; ++b)
    for (int m = 0; m < pr->M; ++m) {
      uint32_t r = draw_word(pr->seed, (uint32_t)b, (uint32_t)m, iter, OR_TAG_PATH);
      I[(size_t)b * pr->M + m] = (int32_t)(((uint64_t)r * (uint64_t)pr->N) >> 32);
    }
}

/* Alg. 1, second step: C = parse_index(Z, I), C[b][m][:] = Z[m][I[b][m]][:]. */
void or_gather_C(const or_problem* pr, const double* Z, const int32_t* I, int32_t P, double* C) {
  for (int b = 0; b < P; ++b)
    for (int m = 0; m < pr->M; ++m) {
      int j = I[(size_t)b * pr->M + m];
      for (int i = 0; i < pr->n; ++i)
        C[((size_t)b * pr->M + m) * pr->n + i] = Z[((size_t)m * pr->N + j) * pr->n + i];
    }
}

/* ------------------------------------------------------------------------- */
/* Eq. 3, Eq. 4 and Def. 2: B-spline control trajectories.                    */
/* ------------------------------------------------------------------------- */

/* Eq. 4 evaluated literally: B_{i,0} is the indicator of [t_i, t_{i+1}) (the
 * interval index `span` is decided by the caller), then the degree is raised
 * by the Cox-de Boor recursion. */
static double cox_de_boor(const double* knots, int i, int p, double t, int span) {
  if (p == 0) return (i == span) ? 1.0 : 0.0;
  double left = 0.0, right = 0.0;
  double dl = knots[i + p] - knots[i];
  double dr = knots[i + p + 1] - knots[i + 1];
  if (dl != 0.0) left = (t - knots[i]) / dl * cox_de_boor(knots, i, p - 1, t, span);
  if (dr != 0.0) right = (knots[i + p + 1] - t) / dr * cox_de_boor(knots, i + 1, p - 1, t, span);
  return left + right;
}

/* Evaluation time of horizon step j (Def. 2, with the valid-span reading). */
double or_bspline_time(int M, int p, int H, int mapping, int j) {
  double K = (double)(M + p + 1);
  if (mapping == OR_TIME_PAPER_LITERAL) return (double)j / (double)H;
  double x = (H > 1) ? (double)p + (double)((M - p) * j) / (double)(H - 1) : (double)p;
  return x / K;
}

/* Def. 2: the basis matrix Bmat[m][j] = B_{m,p}(t_j), m < M, j < H. */
void or_bspline_basis(int M, int p, int H, int mapping, double* Bmat) {
  int nk = M + p + 1;
  double* knots = (double*)malloc(sizeof(double) * (size_t)nk);
  for (int i = 0; i < nk; ++i) knots[i] = (double)i / (double)(M + p + 1);
  for (int j = 0; j < H; ++j) {
    double t = or_bspline_time(M, p, H, mapping, j);
    int span = -1;
    for (int i = 0; i + 1 < nk; ++i)
      if (knots[i] <= t && t < knots[i + 1]) span = i;
    if (mapping == OR_TIME_VALID_SPAN && j == H - 1 && H > 1) span = M - 1; /* closed at t_M */
    for (int m = 0; m < M; ++m) Bmat[(size_t)m * H + j] = cox_de_boor(knots, m, p, t, span);
  }
  free(knots);
}

/* bfloat16 rounding: the nearest number with an 8-bit significand (the
 * exponent range of FP32), ties to the even significand.  Written from that
 * definition: x = f * 2^e with f in [0.5, 1); f * 2^8 is rounded to an integer
 * by rint (round-half-even in the default rounding mode). */
double or_bf16_round(double x) {
  if (x == 0.0 || !isfinite(x)) return x;
  int e;
  double f = frexp(x, &e);
  return ldexp(rint(ldexp(f, 8)), e - 8);
}

/* An operand of the BF16 contraction: the value as FP32, then to BF16. */
static double bf16_operand(double x) { return or_bf16_round((double)(float)x); }

/* Def. 2: U = einsum over the M layers of Bmat and C, U[b][j][i]. */
void or_interp_bspline(const or_problem* pr, const double* C, int32_t P, double* U) {
  double* Bmat = (double*)malloc(sizeof(double) * (size_t)pr->M * pr->H);
  or_bspline_basis(pr->M, pr->degree, pr->H, pr->time_mapping, Bmat);
  for (int b = 0; b < P; ++b)
    for (int j = 0; j < pr->H; ++j)
      for (int i = 0; i < pr->n; ++i) {
        double acc = 0.0;
        for (int m = 0; m < pr->M; ++m) {
          double bm = Bmat[(size_t)m * pr->H + j];
          double cm = C[((size_t)b * pr->M + m) * pr->n + i];
          if (pr->bf16_basis) {
            bm = bf16_operand(bm);
            cm = bf16_operand(cm);
          }
          acc += bm * cm;
        }
        U[((size_t)b * pr->H + j) * pr->n + i] = acc;
      }
  free(Bmat);
}

/* ------------------------------------------------------------------------- */
/* Eqs. 5-7 and Def. 3: Akima-spline control trajectories.                    */
/* ------------------------------------------------------------------------- */

double or_akima_knot(int M, int mapping, int i) {
  return (mapping == OR_TIME_PAPER_LITERAL) ? (double)i / (double)M : (double)i / (double)(M - 1);
}

double or_akima_time(int H, int mapping, int j) {
  if (mapping == OR_TIME_PAPER_LITERAL) return (double)j / (double)H;
  return (H > 1) ? (double)j / (double)(H - 1) : 0.0;
}

/* Eqs. 6-7 for one knot sequence z[0..M-1] at times tk[0..M-1]: writes the
 * coefficients (a, b, c, d) of the M-1 cubic pieces into coef[4*(M-1)].
 * The paper's 1-based indices i map to 0-based i-1 here. */
void or_akima_coeffs(int M, const double* tk, const double* z, double* coef) {
  double m[OR_MAXL * 4 + 8];
  double s[OR_MAXL * 4 + 8];
  /* slopes m_i = (z_{i+1} - z_i)/(t_{i+1} - t_i), i = 1..M-1 */
  for (int i = 1; i <= M - 1; ++i) m[i] = (z[i] - z[i - 1]) / (tk[i] - tk[i - 1]);
  if (M == 2) {
    s[1] = m[1];
    s[2] = m[1];
  } else {
    /* end rules stated under Eq. 6 */
    s[1] = m[1];
    s[M] = m[M - 1];
    s[2] = (m[1] + m[2]) / 2.0;
    s[M - 1] = (m[M - 1] + m[M - 2]) / 2.0;
    /* Eq. 6 for the interior points 3 <= i <= M-2 */
    for (int i = 3; i <= M - 2; ++i) {
      double w1 = fabs(m[i + 1] - m[i]);
      double w2 = fabs(m[i - 1] - m[i - 2]);
      if (w1 + w2 == 0.0)
        s[i] = (m[i - 1] + m[i]) / 2.0;
      else
        s[i] = (w1 * m[i - 1] + w2 * m[i]) / (w1 + w2);
    }
  }
  /* Eq. 7: coefficients of the piece on [t_i, t_{i+1}] */
  for (int i = 1; i <= M - 1; ++i) {
    double h = tk[i] - tk[i - 1];
    double* c = coef + 4 * (i - 1);
    c[0] = z[i - 1];
    c[1] = s[i];
    c[2] = (3.0 * m[i] - 2.0 * s[i] - s[i + 1]) / h;
    c[3] = (s[i] + s[i + 1] - 2.0 * m[i]) / (h * h);
  }
}

/* Eq. 5 at time t: the piece whose left knot is the last knot <= t (clamped to
 * the first and last piece). */
double or_akima_eval(int M, const double* tk, const double* coef, double t) {
  int seg = 0;
  for (int i = 0; i <= M - 2; ++i)
    if (tk[i] <= t) seg = i;
  double dt = t - tk[seg];
  const double* c = coef + 4 * seg;
  return c[3] * dt * dt * dt + c[2] * dt * dt + c[1] * dt + c[0];
}

/* Def. 3: for each path b and control dimension i, Akima through the M
 * waypoints C[b][:][i], evaluated at the H horizon times. */
void or_interp_akima(const or_problem* pr, const double* C, int32_t P, double* U) {
  int M = pr->M;
  double tk[OR_MAXL * 4 + 8], z[OR_MAXL * 4 + 8], coef[4 * (OR_MAXL * 4 + 8)];
  for (int i = 0; i < M; ++i) tk[i] = or_akima_knot(M, pr->time_mapping, i);
  for (int b = 0; b < P; ++b)
    for (int i = 0; i < pr->n; ++i) {
      for (int m = 0; m < M; ++m) z[m] = C[((size_t)b * M + m) * pr->n + i];
      or_akima_coeffs(M, tk, z, coef);
      for (int j = 0; j < pr->H; ++j)
        U[((size_t)b * pr->H + j) * pr->n + i] =
            or_akima_eval(M, tk, coef, or_akima_time(pr->H, pr->time_mapping, j));
    }
}

/* Straight-line interpolation through the waypoints (Sec. 3.1, control path
 * interpolation), with the same knot/time reading as Def. 3. */
void or_interp_linear(const or_problem* pr, const double* C, int32_t P, double* U) {
  int M = pr->M;
  double tk[OR_MAXL * 4 + 8];
  for (int i = 0; i < M; ++i) tk[i] = or_akima_knot(M, pr->time_mapping, i);
  for (int b = 0; b < P; ++b)
    for (int j = 0; j < pr->H; ++j) {
      double t = or_akima_time(pr->H, pr->time_mapping, j);
      int seg = 0;
      for (int k = 0; k <= M - 2; ++k)
        if (tk[k] <= t) seg = k;
      double w = (t - tk[seg]) / (tk[seg + 1] - tk[seg]);
      if (w > 1.0) w = 1.0;
      for (int i = 0; i < pr->n; ++i) {
        double z0 = C[((size_t)b * M + seg) * pr->n + i];
        double z1 = C[((size_t)b * M + seg + 1) * pr->n + i];
        U[((size_t)b * pr->H + j) * pr->n + i] = z0 + w * (z1 - z0);
      }
    }
}

void or_interpolate(const or_problem* pr, const double* C, int32_t P, double* U) {
  if (pr->M == 1) {
    /* a single layer is a constant path */
    for (int b = 0; b < P; ++b)
      for (int j = 0; j < pr->H; ++j)
        for (int i = 0; i < pr->n; ++i)
          U[((size_t)b * pr->H + j) * pr->n + i] = C[(size_t)b * pr->n + i];
    return;
  }
  if (pr->interp == OR_INTERP_BSPLINE) or_interp_bspline(pr, C, P, U);
  else if (pr->interp == OR_INTERP_AKIMA) or_interp_akima(pr, C, P, U);
  else or_interp_linear(pr, C, P, U);
}

/* ------------------------------------------------------------------------- */
/* Alg. 2 local sampling (Sec. 2.1, Eq. of the sampling step).                */
/* ------------------------------------------------------------------------- */

/* Standard normal draws by the Box-Muller transform; one generator call gives
 * the four draws of elements 4q..4q+3 of a candidate's (H x n) row. */
double or_standard_normal(uint64_t seed, uint32_t iter, uint32_t b, uint32_t e) {
  uint32_t q = e >> 2;
  uint32_t ctr[4] = {b, q, iter, OR_TAG_LOCAL};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t w[4];
  or_philox4x32_10(ctr, key, w);
  int pair = (e & 3u) >> 1;
  double u1 = ((double)(w[2 * pair] >> 8) + 1.0) * (1.0 / 16777216.0); /* (0, 1] */
  double u2 = (double)(w[2 * pair + 1] >> 8) * (1.0 / 16777216.0);     /* [0, 1) */
  double radius = sqrt(-2.0 * log(u1));
  double angle = 2.0 * M_PI * u2;
  return (e & 1u) ? radius * sin(angle) : radius * cos(angle);
}

/* U_local[b] ~ N(mu, diag(sigma^2)) for the first L = B-P-1 candidates. */
void or_local_samples(const or_problem* pr, uint32_t iter, const double* mu, const double* sigma,
                      int32_t L, double* UL) {
  for (int b = 0; b < L; ++b)
    for (int j = 0; j < pr->H; ++j)
      for (int i = 0; i < pr->n; ++i) {
        uint32_t e = (uint32_t)(j * pr->n + i);
        double eps = or_standard_normal(pr->seed, iter, (uint32_t)b, e);
        UL[((size_t)b * pr->H + j) * pr->n + i] = mu[j * pr->n + i] + sigma[j * pr->n + i] * eps;
      }
}

/* Alg. 2 stacking: rows [0, L) local, [L, L+P) graph, row B-1 the nominal mu,
 * then every control clamped to the box. */
void or_stack_clamp(const or_problem* pr, const double* UL, const double* UG, const double* mu,
                    double* U) {
  int32_t P = pr->P, L = pr->B - P - 1;
  size_t row = (size_t)pr->H * pr->n;
  if (L > 0) memcpy(U, UL, sizeof(double) * row * (size_t)L);
  if (P > 0) memcpy(U + row * (size_t)L, UG, sizeof(double) * row * (size_t)P);
  memcpy(U + row * (size_t)(pr->B - 1), mu, sizeof(double) * row);
  for (int b = 0; b < pr->B; ++b)
    for (int j = 0; j < pr->H; ++j)
      for (int i = 0; i < pr->n; ++i) {
        double* u = &U[((size_t)b * pr->H + j) * pr->n + i];
        if (*u < pr->u_min[i]) *u = pr->u_min[i];
        if (*u > pr->u_max[i]) *u = pr->u_max[i];
      }
}

/* ------------------------------------------------------------------------- */
/* Domain randomisation (Sec. 4, practical settings).                         */
/* ------------------------------------------------------------------------- */

/* Scale factor for parameter slot `slot` of model `unit` (a candidate in the
 * per-sample mode, one of R shared models in the shared mode). */
double or_dr_scale(const or_problem* pr, uint32_t iter, uint32_t unit, uint32_t slot) {
  if (pr->dr_mode == OR_DR_NONE) return 1.0;
  uint32_t tag = (pr->dr_mode == OR_DR_SHARED) ? OR_TAG_PARAM_MODEL : OR_TAG_PARAM_SAMPLE;
  uint32_t r = draw_word(pr->seed, unit, slot, iter, tag);
  return pr->dr_lo + (pr->dr_hi - pr->dr_lo) * unit_uniform(r);
}

/* ------------------------------------------------------------------------- */
/* Dynamics f(x, u) and costs (Eq. 2).                                        */
/* ------------------------------------------------------------------------- */

/* Point mass in k = n dimensions; state x = (p, v); control u is acceleration
 * times the actuation gain; semi-implicit Euler. */
static void pm_step(const or_problem* pr, const double* gain, double* x, const double* u) {
  int k = pr->n;
  for (int a = 0; a < k; ++a) {
    x[k + a] = x[k + a] + pr->dt * gain[a] * u[a];
    x[a] = x[a] + pr->dt * x[k + a];
  }
}

static double pm_state_cost(const or_problem* pr, const double* x) {
  int k = pr->n;
  double dist2 = 0.0;
  for (int a = 0; a < k; ++a) dist2 += (x[a] - pr->target[a]) * (x[a] - pr->target[a]);
  double pen = 0.0;
  for (int o = 0; o < pr->n_obs; ++o) {
    double d2 = 0.0;
    for (int a = 0; a < k; ++a) d2 += (x[a] - pr->obs_c[o][a]) * (x[a] - pr->obs_c[o][a]);
    double depth = pr->obs_r[o] - sqrt(d2);
    if (depth > 0.0) pen += depth;
  }
  return pr->w_target * dist2 + pr->w_obs * pen;
}

static double pm_stage_cost(const or_problem* pr, const double* x, const double* u) {
  double uu = 0.0;
  for (int a = 0; a < pr->n; ++a) uu += u[a] * u[a];
  return pm_state_cost(pr, x) + pr->w_ctrl * uu;
}

/* Planar serial chain, textbook recursive Newton-Euler in the world frame.
 * Joint j (0-based) connects link j-1 (the fixed base for j = 0) to link j;
 * q are relative joint angles, absolute angle phi_j = q_0 + ... + q_j.
 * Links are uniform thin rods: COM at l/2, inertia m l^2/12.  Gravity acts
 * along -y.  Returns the joint torques tau = ID(q, qd, qdd). */
static void chain_rnea(int nl, const double* mass, const double* len, double g, const double* q,
                       const double* qd, const double* qdd, double* tau) {
  double phi = 0.0, w = 0.0, al = 0.0;
  double ox = 0.0, oy = 0.0, aox = 0.0, aoy = 0.0; /* joint origin and its acceleration */
  double Fx[OR_MAXL], Fy[OR_MAXL], rcx[OR_MAXL], rcy[OR_MAXL], rnx[OR_MAXL], rny[OR_MAXL];
  double alpha[OR_MAXL];
  for (int j = 0; j < nl; ++j) {
    phi += q[j];
    w += qd[j];
    al += qdd[j];
    double ex = cos(phi), ey = sin(phi);
    double h = 0.5 * len[j];
    /* COM acceleration: a_o + al x r - w^2 r */
    double acx = aox - al * h * ey - w * w * h * ex;
    double acy = aoy + al * h * ex - w * w * h * ey;
    Fx[j] = mass[j] * acx;
    Fy[j] = mass[j] * (acy + g);
    rcx[j] = h * ex; rcy[j] = h * ey;               /* COM relative to joint j */
    rnx[j] = len[j] * ex; rny[j] = len[j] * ey;     /* joint j+1 relative to joint j */
    alpha[j] = al;
    aox = aox - al * len[j] * ey - w * w * len[j] * ex;
    aoy = aoy + al * len[j] * ex - w * w * len[j] * ey;
    ox += rnx[j]; oy += rny[j];
  }
  double fx = 0.0, fy = 0.0, nz = 0.0; /* force and moment passed from link j+1 */
  for (int j = nl - 1; j >= 0; --j) {
    double inertia = mass[j] * len[j] * len[j] / 12.0;
    double n_new = inertia * alpha[j] + nz + (rcx[j] * Fy[j] - rcy[j] * Fx[j]) +
                   (rnx[j] * fy - rny[j] * fx);
    fx = Fx[j] + fx;
    fy = Fy[j] + fy;
    nz = n_new;
    tau[j] = nz;
  }
  (void)ox; (void)oy;
}

/* Solve the symmetric positive definite system A x = b by Cholesky. */
static int cholesky_solve(int n, double* A, double* b, double* x) {
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
    if (!(s > 0.0)) return -1;
    A[j * n + j] = sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = t / A[j * n + j];
    }
  }
  for (int i = 0; i < n; ++i) {
    double t = b[i];
    for (int k = 0; k < i; ++k) t -= A[i * n + k] * x[k];
    x[i] = t / A[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double t = x[i];
    for (int k = i + 1; k < n; ++k) t -= A[k * n + i] * x[k];
    x[i] = t / A[i * n + i];
  }
  return 0;
}

/* Forward dynamics of the chain: mass matrix columns from unit accelerations
 * of the inverse dynamics (gravity and velocity off), bias from the inverse
 * dynamics at zero acceleration, then qdd = M^-1 (tau - bias). */
int or_chain_forward_dynamics(int nl, const double* mass, const double* len, double g,
                              const double* q, const double* qd, const double* tau, double* qdd) {
  double Mm[OR_MAXL * OR_MAXL], bias[OR_MAXL], zero[OR_MAXL], e[OR_MAXL], col[OR_MAXL];
  double rhs[OR_MAXL];
  for (int j = 0; j < nl; ++j) zero[j] = 0.0;
  chain_rnea(nl, mass, len, g, q, qd, zero, bias);
  for (int c = 0; c < nl; ++c) {
    for (int j = 0; j < nl; ++j) e[j] = (j == c) ? 1.0 : 0.0;
    chain_rnea(nl, mass, len, 0.0, q, zero, e, col);
    for (int r = 0; r < nl; ++r) Mm[r * nl + c] = col[r];
  }
  for (int j = 0; j < nl; ++j) rhs[j] = tau[j] - bias[j];
  return cholesky_solve(nl, Mm, rhs, qdd);
}

/* Mechanical energy of the chain (kinetic + potential), used by the tests. */
double or_chain_energy(int nl, const double* mass, const double* len, double g, const double* q,
                       const double* qd) {
  double phi = 0.0, w = 0.0, ox = 0.0, oy = 0.0, vox = 0.0, voy = 0.0, E = 0.0;
  for (int j = 0; j < nl; ++j) {
    phi += q[j];
    w += qd[j];
    double ex = cos(phi), ey = sin(phi), h = 0.5 * len[j];
    double vcx = vox - w * h * ey, vcy = voy + w * h * ex;
    double cy = oy + h * ey;
    E += 0.5 * mass[j] * (vcx * vcx + vcy * vcy) + 0.5 * (mass[j] * len[j] * len[j] / 12.0) * w * w;
    E += mass[j] * g * cy;
    vox -= w * len[j] * ey; voy += w * len[j] * ex;
    ox += len[j] * ex; oy += len[j] * ey;
  }
  (void)ox;
  return E;
}

static void chain_tip(int nl, const double* len, const double* q, double* tip) {
  double phi = 0.0, x = 0.0, y = 0.0;
  for (int j = 0; j < nl; ++j) {
    phi += q[j];
    x += len[j] * cos(phi);
    y += len[j] * sin(phi);
  }
  tip[0] = x; tip[1] = y;
}

static double chain_reach_cost(const or_problem* pr, const double* x) {
  double tip[2];
  chain_tip(pr->n_links, pr->length, x, tip);
  double dx = tip[0] - pr->target[0], dy = tip[1] - pr->target[1];
  return pr->w_target * (dx * dx + dy * dy);
}

/* One semi-implicit Euler step of the chain: qd += dt qdd; q += dt qd. */
static int chain_step(const or_problem* pr, const double* mass, double* x, const double* u) {
  int nl = pr->n_links;
  double qdd[OR_MAXL];
  int rc = or_chain_forward_dynamics(nl, mass, pr->length, pr->gravity, x, x + nl, u, qdd);
  for (int j = 0; j < nl; ++j) {
    x[nl + j] = x[nl + j] + pr->dt * qdd[j];
    x[j] = x[j] + pr->dt * x[nl + j];
  }
  return rc;
}

/* Legged model: a planar chain with a floating base.  Generalised
 * coordinates are (x_b, y_b, phi_0, q_1..q_{L-1}): the proximal end of link 0,
 * its absolute angle, then the relative joint angles.  The oracle writes it as
 * a chain whose first two joints are massless prismatic joints along x and y,
 * so the same recursive Newton-Euler pass applies with joint types. */
static void legged_rnea(int nl, const double* mass, const double* len, double g, const double* q,
                        const double* qd, const double* qdd, const double* fext_x,
                        const double* fext_y, double* tau) {
  /* q[0], q[1]: base translation; q[2..]: angles (first absolute, rest relative) */
  double aox = qdd[0], aoy = qdd[1];
  double phi = 0.0, w = 0.0, al = 0.0;
  double Fx[OR_MAXL], Fy[OR_MAXL], rcx[OR_MAXL], rcy[OR_MAXL], rnx[OR_MAXL], rny[OR_MAXL];
  double alpha[OR_MAXL];
  for (int j = 0; j < nl; ++j) {
    phi += q[2 + j];
    w += qd[2 + j];
    al += qdd[2 + j];
    double ex = cos(phi), ey = sin(phi), h = 0.5 * len[j];
    double acx = aox - al * h * ey - w * w * h * ex;
    double acy = aoy + al * h * ex - w * w * h * ey;
    Fx[j] = mass[j] * acx;
    Fy[j] = mass[j] * (acy + g);
    rcx[j] = h * ex; rcy[j] = h * ey;
    rnx[j] = len[j] * ex; rny[j] = len[j] * ey;
    alpha[j] = al;
    aox = aox - al * len[j] * ey - w * w * len[j] * ex;
    aoy = aoy + al * len[j] * ex - w * w * len[j] * ey;
  }
  /* external contact forces act at the distal end of each link (index j+1)
   * and at the proximal end of link 0 (index 0); they enter with a minus
   * sign as forces the joints need not supply. */
  double fx = 0.0, fy = 0.0, nz = 0.0;
  for (int j = nl - 1; j >= 0; --j) {
    double inertia = mass[j] * len[j] * len[j] / 12.0;
    double fdx = fx - fext_x[j + 1], fdy = fy - fext_y[j + 1]; /* force on link j+1 side */
    double n_new = inertia * alpha[j] + nz + (rcx[j] * Fy[j] - rcy[j] * Fx[j]) +
                   (rnx[j] * fdy - rny[j] * fdx);
    fx = Fx[j] + fdx;
    fy = Fy[j] + fdy;
    nz = n_new;
    tau[2 + j] = nz;
  }
  /* prismatic base joints carry the total force, minus the contact at the base point */
  tau[0] = fx - fext_x[0];
  tau[1] = fy - fext_y[0];
}

/* Contact points: base point (index 0) and the distal end of every link.
 * Ground y = 0; spring-damper normal force and smoothed Coulomb friction. */
static void legged_contacts(const or_problem* pr, double mu_scale, const double* q,
                            const double* qd, double* fx, double* fy) {
  int nl = pr->n_links;
  double px = q[0], py = q[1], vx = qd[0], vy = qd[1], phi = 0.0, w = 0.0;
  for (int c = 0; c <= nl; ++c) {
    double f_n = 0.0;
    if (py < 0.0) {
      f_n = pr->k_contact * (-py) - pr->c_contact * vy;
      if (f_n < 0.0) f_n = 0.0;
    }
    fx[c] = -pr->mu_friction * mu_scale * f_n * tanh(vx / pr->v_slip);
    fy[c] = f_n;
    if (c < nl) {
      phi += q[2 + c];
      w += qd[2 + c];
      double ex = cos(phi), ey = sin(phi);
      px += pr->length[c] * ex; py += pr->length[c] * ey;
      vx -= w * pr->length[c] * ey; vy += w * pr->length[c] * ex;
    }
  }
}

int or_legged_forward_dynamics(const or_problem* pr, const double* mass, double mu_scale,
                               const double* q, const double* qd, const double* tau_joint,
                               double* qdd) {
  int nl = pr->n_links, nd = nl + 2;
  double Mm[(OR_MAXL + 2) * (OR_MAXL + 2)], bias[OR_MAXL + 2], zero[OR_MAXL + 2];
  double e[OR_MAXL + 2], col[OR_MAXL + 2], rhs[OR_MAXL + 2], tau[OR_MAXL + 2];
  double fx[OR_MAXL + 1], fy[OR_MAXL + 1], zf[OR_MAXL + 1];
  for (int j = 0; j < nd; ++j) zero[j] = 0.0;
  for (int c = 0; c <= nl; ++c) zf[c] = 0.0;
  legged_contacts(pr, mu_scale, q, qd, fx, fy);
  legged_rnea(nl, mass, pr->length, pr->gravity, q, qd, zero, fx, fy, bias);
  for (int c = 0; c < nd; ++c) {
    for (int j = 0; j < nd; ++j) e[j] = (j == c) ? 1.0 : 0.0;
    legged_rnea(nl, mass, pr->length, 0.0, q, zero, e, zf, zf, col);
    for (int r = 0; r < nd; ++r) Mm[r * nd + c] = col[r];
  }
  /* the base (x, y, phi_0) is unactuated; joint torques drive q_1..q_{L-1} */
  tau[0] = tau[1] = tau[2] = 0.0;
  for (int j = 1; j < nl; ++j) tau[2 + j] = tau_joint[j - 1];
  for (int j = 0; j < nd; ++j) rhs[j] = tau[j] - bias[j];
  return cholesky_solve(nd, Mm, rhs, qdd);
}

static int legged_step(const or_problem* pr, const double* mass, double mu_scale, double* x,
                       const double* u) {
  int nd = pr->n_links + 2;
  double qdd[OR_MAXL + 2];
  int rc = or_legged_forward_dynamics(pr, mass, mu_scale, x, x + nd, u, qdd);
  for (int j = 0; j < nd; ++j) {
    x[nd + j] = x[nd + j] + pr->dt * qdd[j];
    x[j] = x[j] + pr->dt * x[nd + j];
  }
  return rc;
}

/* Walker-like cost (Sec. A task details, Walker): torso height, pitch and
 * forward velocity of link 0's proximal end, plus a control penalty. */
static double legged_state_cost(const or_problem* pr, const double* x) {
  int nd = pr->n_links + 2;
  double h = x[1], pitch = x[2], v = x[nd + 0];
  double dh = h - pr->target[0], dv = v - pr->target[1], dp = pitch - pr->target[2];
  return pr->w_height * dh * dh + pr->w_pitch * dp * dp + pr->w_vel * dv * dv;
}

/* Eq. 2 for one candidate and one model: J = sum_t c(x_t, u_t) + c_T(x_T). */
static double rollout_one(const or_problem* pr, uint32_t iter, const double* x0, const double* Ub,
                          uint32_t dr_unit, double* states) {
  double x[2 * (OR_MAXL + 2) + 2 * OR_MAXN];
  double mass[OR_MAXL], gain[OR_MAXN];
  double mu_scale = 1.0;
  int d = pr->d;
  for (int a = 0; a < d; ++a) x[a] = x0[a];
  if (states) memcpy(states, x, sizeof(double) * (size_t)d);
  if (pr->dyn == OR_DYN_POINTMASS) {
    for (int a = 0; a < pr->n; ++a) gain[a] = or_dr_scale(pr, iter, dr_unit, (uint32_t)a);
  } else if (pr->dyn == OR_DYN_CHAIN) {
    for (int j = 0; j < pr->n_links; ++j)
      mass[j] = pr->mass[j] * or_dr_scale(pr, iter, dr_unit, (uint32_t)j);
  } else {
    for (int j = 0; j < pr->n_links; ++j)
      mass[j] = pr->mass[j] * or_dr_scale(pr, iter, dr_unit, (uint32_t)j);
    mu_scale = or_dr_scale(pr, iter, dr_unit, (uint32_t)pr->n_links);
  }
  double J = 0.0;
  for (int t = 0; t < pr->H; ++t) {
    const double* u = Ub + (size_t)t * pr->n;
    if (pr->dyn == OR_DYN_POINTMASS) {
      J += pm_stage_cost(pr, x, u);
      pm_step(pr, gain, x, u);
    } else if (pr->dyn == OR_DYN_CHAIN) {
      double uu = 0.0;
      for (int a = 0; a < pr->n; ++a) uu += u[a] * u[a];
      J += chain_reach_cost(pr, x) + pr->w_ctrl * uu;
      if (chain_step(pr, mass, x, u) != 0) return INFINITY;
    } else {
      double uu = 0.0;
      for (int a = 0; a < pr->n; ++a) uu += u[a] * u[a];
      J += legged_state_cost(pr, x) + pr->w_ctrl * uu;
      if (legged_step(pr, mass, mu_scale, x, u) != 0) return INFINITY;
    }
    if (states) memcpy(states + (size_t)(t + 1) * d, x, sizeof(double) * (size_t)d);
  }
  if (pr->dyn == OR_DYN_POINTMASS) J += pr->w_term * pm_state_cost(pr, x);
  else if (pr->dyn == OR_DYN_CHAIN) J += pr->w_term * chain_reach_cost(pr, x);
  else J += pr->w_term * legged_state_cost(pr, x);
  return J;
}

/* Alg. 2 batch rollout for candidates [row0, row0+nrows): cost s_b; with R
 * shared randomised models the cost is averaged over them (Sec. 4). */
void or_rollout_costs(const or_problem* pr, uint32_t iter, const double* x0, const double* U,
                      int32_t row0, int32_t nrows, double* cost) {
  size_t row = (size_t)pr->H * pr->n;
  for (int r = 0; r < nrows; ++r) {
    int b = row0 + r;
    const double* Ub = U + row * (size_t)r;
    if (pr->dr_mode == OR_DR_SHARED) {
      double acc = 0.0;
      for (int k = 0; k < pr->R; ++k) acc += rollout_one(pr, iter, x0, Ub, (uint32_t)k, NULL);
      cost[r] = acc / (double)pr->R;
    } else {
      cost[r] = rollout_one(pr, iter, x0, Ub, (uint32_t)b, NULL);
    }
  }
}

/* The same costs with the candidates split into `threads` contiguous chunks,
 * one POSIX thread per chunk.  Each candidate's cost is computed exactly as
 * above (candidates are independent until the selection), so the result does
 * not depend on the thread count; this only spreads the slow FP64 rollouts
 * over the host's cores. */
typedef struct {
  const or_problem* pr;
  uint32_t iter;
  const double* x0;
  const double* U;
  int32_t row0, nrows;
  double* cost;
} or_chunk;

static void* rollout_chunk(void* arg) {
  or_chunk* c = (or_chunk*)arg;
  or_rollout_costs(c->pr, c->iter, c->x0, c->U, c->row0, c->nrows, c->cost);
  return NULL;
}

void or_rollout_costs_threads(const or_problem* pr, uint32_t iter, const double* x0,
                              const double* U, int32_t row0, int32_t nrows, double* cost,
                              int32_t threads) {
  if (threads > nrows) threads = nrows;
  if (threads <= 1) {
    or_rollout_costs(pr, iter, x0, U, row0, nrows, cost);
    return;
  }
  size_t row = (size_t)pr->H * pr->n;
  pthread_t* tid = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
  or_chunk* ch = (or_chunk*)malloc(sizeof(or_chunk) * (size_t)threads);
  int* started = (int*)calloc((size_t)threads, sizeof(int));
  int32_t at = 0;
  for (int k = 0; k < threads; ++k) {
    int32_t cnt = nrows / threads + (k < nrows % threads ? 1 : 0);
    ch[k].pr = pr; ch[k].iter = iter; ch[k].x0 = x0;
    ch[k].U = U + row * (size_t)at;
    ch[k].row0 = row0 + at; ch[k].nrows = cnt;
    ch[k].cost = cost + at;
    at += cnt;
    started[k] = pthread_create(&tid[k], NULL, rollout_chunk, &ch[k]) == 0;
    if (!started[k]) rollout_chunk(&ch[k]); /* no thread to be had: run it here */
  }
  for (int k = 0; k < threads; ++k)
    if (started[k]) pthread_join(tid[k], NULL);
  free(started); free(ch); free(tid);
}

/* State trajectory (H+1) x d of candidate b under its own randomised model. */
double or_rollout_states(const or_problem* pr, uint32_t iter, const double* x0, const double* Ub,
                         int32_t b, double* states) {
  return rollout_one(pr, iter, x0, Ub, (uint32_t)b, states);
}

/* ------------------------------------------------------------------------- */
/* Alg. 2 elite selection and the modified CEM update.                       */
/* ------------------------------------------------------------------------- */

typedef struct { double cost; int32_t idx; } or_key;

static int key_cmp(const void* a, const void* b) {
  const or_key* x = (const or_key*)a;
  const or_key* y = (const or_key*)b;
  if (x->cost < y->cost) return -1;
  if (x->cost > y->cost) return 1;
  return (x->idx < y->idx) ? -1 : (x->idx > y->idx);
}

/* Top-E: indices of the E smallest costs, ascending by (cost, index). */
void or_top_e(const double* cost, int32_t B, int32_t E, int32_t* elite) {
  or_key* keys = (or_key*)malloc(sizeof(or_key) * (size_t)B);
  for (int b = 0; b < B; ++b) {
    double c = cost[b];
    if (isnan(c)) c = INFINITY;
    keys[b].cost = c;
    keys[b].idx = b;
  }
  qsort(keys, (size_t)B, sizeof(or_key), key_cmp);
  for (int k = 0; k < E; ++k) elite[k] = keys[k].idx;
  free(keys);
}

/* Softmax weights over the elite costs, w_k proportional to exp(-s_k/lambda),
 * computed after subtracting the best cost (the weights are unchanged). */
void or_softmax_weights(const double* cost, const int32_t* elite, int32_t E, double lambda,
                        double* w) {
  double smin = cost[elite[0]];
  if (isnan(smin)) smin = INFINITY;
  if (isinf(smin)) {
    for (int k = 0; k < E; ++k) w[k] = 1.0 / (double)E;
    return;
  }
  double total = 0.0;
  for (int k = 0; k < E; ++k) {
    double c = cost[elite[k]];
    if (isnan(c)) c = INFINITY;
    w[k] = exp(-(c - smin) / lambda);
    total += w[k];
  }
  for (int k = 0; k < E; ++k) w[k] /= total;
}

/* Alg. 2 update: mu' = w U_E, sigma' = max(sqrt(sum_k w_k (U_k - mu')^2), sigma_m),
 * then mu <- mu' + alpha (mu - mu'), sigma <- sigma' + alpha (sigma - sigma').
 * With update_rule = plain CEM the Sec. 2.1 CEM update is used instead:
 * unweighted mean, 1/(E-1) variance, smoothing alpha*old + (1-alpha)*new.
 * u* = U[elite[0]][0][:]. */
void or_elite_update(const or_problem* pr, const double* U, const double* cost,
                     const int32_t* elite, double* mu, double* sigma, double* ustar) {
  int E = pr->E, H = pr->H, n = pr->n;
  size_t row = (size_t)H * n;
  double* w = (double*)malloc(sizeof(double) * (size_t)E);
  if (pr->update_rule == OR_UPDATE_SOFTMAX) or_softmax_weights(cost, elite, E, pr->lambda, w);
  for (int e = 0; e < H * n; ++e) {
    if (pr->update_rule == OR_UPDATE_SOFTMAX) {
      double m1 = 0.0;
      for (int k = 0; k < E; ++k) m1 += w[k] * U[row * (size_t)elite[k] + e];
      double v = 0.0;
      for (int k = 0; k < E; ++k) {
        double dlt = U[row * (size_t)elite[k] + e] - m1;
        v += w[k] * dlt * dlt;
      }
      double s1 = sqrt(v);
      if (s1 < pr->sigma_min) s1 = pr->sigma_min;
      mu[e] = m1 + pr->alpha * (mu[e] - m1);
      sigma[e] = s1 + pr->alpha * (sigma[e] - s1);
    } else {
      double m1 = 0.0;
      for (int k = 0; k < E; ++k) m1 += U[row * (size_t)elite[k] + e];
      m1 /= (double)E;
      double v = 0.0;
      for (int k = 0; k < E; ++k) {
        double dlt = U[row * (size_t)elite[k] + e] - m1;
        v += dlt * dlt;
      }
      double s1 = (E > 1) ? sqrt(v / (double)(E - 1)) : 0.0;
      mu[e] = pr->alpha * mu[e] + (1.0 - pr->alpha) * m1;
      sigma[e] = pr->alpha * sigma[e] + (1.0 - pr->alpha) * s1;
    }
  }
  for (int i = 0; i < n; ++i) ustar[i] = U[row * (size_t)elite[0] + i];
  free(w);
}

/* Warm start between control steps: shift mu and sigma k steps earlier and
 * repeat the last row (the paper is silent on this). */
void or_shift(int H, int n, int k, double* mu, double* sigma) {
  if (k <= 0) return;
  for (int t = 0; t < H; ++t) {
    int src = t + k < H ? t + k : H - 1;
    for (int i = 0; i < n; ++i) {
      mu[t * n + i] = mu[src * n + i];
      sigma[t * n + i] = sigma[src * n + i];
    }
  }
}

/* ------------------------------------------------------------------------- */
/* One full planner iteration (Alg. 2 loop body).                             */
/* ------------------------------------------------------------------------- */

int or_plan_iteration_threads(const or_problem* pr, uint32_t iter, const double* x0, double* mu,
                              double* sigma, double* U_out, double* cost_out, int32_t* elite_out,
                              double* ustar, int32_t threads) {
  int32_t P = pr->P, L = pr->B - P - 1;
  size_t row = (size_t)pr->H * pr->n;
  double* Z = (double*)malloc(sizeof(double) * (size_t)pr->M * pr->N * pr->n);
  int32_t* I = (int32_t*)malloc(sizeof(int32_t) * (size_t)(P > 0 ? P : 1) * pr->M);
  double* C = (double*)malloc(sizeof(double) * (size_t)(P > 0 ? P : 1) * pr->M * pr->n);
  double* UG = (double*)malloc(sizeof(double) * row * (size_t)(P > 0 ? P : 1));
  double* UL = (double*)malloc(sizeof(double) * row * (size_t)(L > 0 ? L : 1));
  double* U = U_out ? U_out : (double*)malloc(sizeof(double) * row * (size_t)pr->B);
  double* cost = cost_out ? cost_out : (double*)malloc(sizeof(double) * (size_t)pr->B);
  int32_t* elite = elite_out ? elite_out : (int32_t*)malloc(sizeof(int32_t) * (size_t)pr->E);
  /* tensor sampling */
  or_graph_Z(pr, iter, Z);
  or_path_indices(pr, iter, P, I);
  or_gather_C(pr, Z, I, P, C);
  or_interpolate(pr, C, P, UG);
  /* local sampling, stacking */
  or_local_samples(pr, iter, mu, sigma, L, UL);
  or_stack_clamp(pr, UL, UG, mu, U);
  /* rollout, cost, elites, update */
  or_rollout_costs_threads(pr, iter, x0, U, 0, pr->B, cost, threads);
  or_top_e(cost, pr->B, pr->E, elite);
  or_elite_update(pr, U, cost, elite, mu, sigma, ustar);
  free(Z); free(I); free(C); free(UG); free(UL);
  if (!U_out) free(U);
  if (!cost_out) free(cost);
  if (!elite_out) free(elite);
  return 0;
}

int or_plan_iteration(const or_problem* pr, uint32_t iter, const double* x0, double* mu,
                      double* sigma, double* U_out, double* cost_out, int32_t* elite_out,
                      double* ustar) {
  return or_plan_iteration_threads(pr, iter, x0, mu, sigma, U_out, cost_out, elite_out, ustar, 1);
}

/* Cost-entropy diagnostic of Sec. 4.1 with the sign read as exp(-J/lambda). */
double or_cost_entropy(const double* cost, int32_t B, double lambda) {
  double cmin = INFINITY;
  for (int b = 0; b < B; ++b) if (cost[b] < cmin) cmin = cost[b];
  double z = 0.0;
  for (int b = 0; b < B; ++b) z += exp(-(cost[b] - cmin) / lambda);
  double h = 0.0;
  for (int b = 0; b < B; ++b) {
    double p = exp(-(cost[b] - cmin) / lambda) / z;
    if (p > 0.0) h -= p * log(p);
  }
  return h;
}
