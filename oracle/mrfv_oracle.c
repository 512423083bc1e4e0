/*
 * mrfv_oracle.c -- plain, slow CPU oracle of the adaptive multiresolution
 * finite-volume method for the compressible Euler equations
 * (Deiterding, Domingues, Gomes, Schneider, arXiv:1603.05211).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the bench may load this library.  It shares no code, header,
 * table or helper with the CUDA path.  It is compiled with -ffp-contract=off so
 * every floating-point operation is rounded where the source says it is.
 *
 * Data model: every level l = 0..L is a dense array of N_l^d cells per
 * variable (layout [v][cell], cell = i + n0*(j + n1*k)) plus a dense byte map
 * of which 8^d-cell blocks exist.  Cells of absent blocks hold NaN, so any read
 * of an absent value poisons the result and shows up in the tests.
 *
 * What each part follows:
 *   - Euler equations, ideal gas, gamma = 1.4 .............. Section 2, Eqs. 2.1-2.3
 *   - cell averages, dQ/dt = -F(Q) ........................ Section 2 (FV semi-discretisation)
 *   - MUSCL, van Albada limiter, AUSM+ flux, RK2 midpoint .. Section 2 (MR scheme paragraph)
 *   - MUSCL-Hancock, Minmod, AUSMDV flux (scheme 1) ....... Section 2 (AMR scheme paragraph), Sec. 4.2
 *   - projection / 3rd-order prediction / details / eps ... Section 2.1
 *   - refinement by one level, gradedness, coarsening ..... Section 2.1 (three basic operations)
 *   - virtual leaves / conservative coarse-fine fluxes ..... Section 2.1, Fig. 1
 *   - level-dependent time steps, time interpolation ....... Section 2.1 (MRLT), Section 2.2, Fig. 2
 *   - flux correction at refinement boundaries ............. Section 2.2, Fig. 2
 *   - scaled-gradient flags + one-cell buffer, clustering .. Section 2.2 (refinement indicators)
 *   - Richardson estimate as an additional indicator ....... Section 2.2 (refinement indicators)
 *   - L1 error by projection to the finest level .......... Section 3
 * Readings where the paper is silent are stated beside the code that takes them.
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OMAXL 12
#define OB 8 /* cells per block edge */
#define OG OMAXL /* geometry slot of the scratch grid */

enum { O_BC_TRANSMISSIVE = 0, O_BC_PERIODIC = 1 };
enum { O_CRIT_MR = 0, O_CRIT_GRAD = 1 };
enum { O_IC_QUADRANTS = 0, O_IC_ELLIPSOID = 1, O_IC_SHOCKTUBE = 2, O_IC_UNIFORM = 3,
       O_IC_WAVE = 4, O_IC_ROTATED_ELLIPSOID = 5 };

enum { O_SCHEME_MUSCL_RK2 = 0, O_SCHEME_HANCOCK = 1 };
enum { O_CLUSTER_ROWS = 0, O_CLUSTER_BR = 1 };

typedef struct {
  int dim, nv, L, bc;
  int scheme;         /* O_SCHEME_*: the MR scheme (default) or the AMR scheme of Section 2 */
  int clustering;     /* O_CLUSTER_*: clustering of gradient flags (Section 2.2) */
  double eps_p;       /* > 0: the gradient criterion also tests pressure (Section 4.2) */
  int lts_remesh;     /* level-dependent steps: remesh the finer levels inside the recursion (Fig. 2)
                         with this criterion and these parameters */
  int rm_crit, rm_precision;
  double rm_eps, rm_epsw, rm_eta;
  double eps_r;       /* > 0: the gradient criterion also flags by the Richardson estimate (Section 2.2) */
  double rich_dt;     /* step of the last orc_step (finest-level step when rich_lts) */
  int rich_lts;
  long rich_bad;      /* Richardson estimates on existing blocks that came out non-finite */
  double gamma;
  double lo[3], hi[3];
  /* geometry; entry OG (= OMAXL) describes a scratch grid (the level coarsened by 2
     of the Richardson estimate) so that the level functions run on it too */
  int nb[OMAXL + 1][3];   /* blocks per dimension (1 in unused dimensions) */
  int n[OMAXL + 1][3];    /* cells per dimension */
  long ncell[OMAXL + 1], nblk[OMAXL + 1];
  double dx[OMAXL + 1][3];
  uint8_t *ex[OMAXL]; /* block exists */
  double *q[OMAXL];   /* state Q^n, [v][cell] */
  double *qs[OMAXL];  /* RK stage state Q* */
  double *q0[OMAXL];  /* state at the start of the level's own step (local time stepping) */
  double *rc[OMAXL];  /* coarse-role flux record: dt*F on [side][dir][v][cell] */
  double *rf[OMAXL];  /* fine-role flux record, summed over the sub-steps of the parent step */
  uint8_t *sig[OMAXL];      /* last analysis: block significant / flagged */
  double *maxdet[OMAXL];    /* last analysis: block max normalised detail */
  double scale[5];          /* last analysis: normalisation s_v */
} orc;

/* ------------------------------------------------------------------------ */
/* indexing                                                                   */

static long cidx(const orc *o, int l, int i, int j, int k) {
  return (long)i + (long)o->n[l][0] * ((long)j + (long)o->n[l][1] * (long)k);
}
static long bidx(const orc *o, int l, int bi, int bj, int bk) {
  return (long)bi + (long)o->nb[l][0] * ((long)bj + (long)o->nb[l][1] * (long)bk);
}
/* boundary handling of a cell coordinate: transmissive = nearest interior cell
   (zero-gradient copy into every ghost layer), periodic = wrap. */
static int bc_cell(const orc *o, int l, int d, int i) {
  int N = o->n[l][d];
  if (d >= o->dim) return 0;
  if (o->bc == O_BC_PERIODIC) { i %= N; if (i < 0) i += N; return i; }
  return i < 0 ? 0 : (i >= N ? N - 1 : i);
}
/* neighbouring block coordinate, or -1 when it lies outside a transmissive domain */
static void apply_need(orc *o, uint8_t **need, int lfrom);
static void remesh_amr(orc *o, int l0, double th);
static void remesh_mr(orc *o, int l0, double th);
static void close_and_nest(orc *o, uint8_t **need, int l0);

static int bc_block(const orc *o, int l, int d, int b) {
  int N = o->nb[l][d];
  if (d >= o->dim) return b == 0 ? 0 : -1;
  if (o->bc == O_BC_PERIODIC) { b %= N; if (b < 0) b += N; return b; }
  return (b < 0 || b >= N) ? -1 : b;
}
static int block_exists(const orc *o, int l, int bi, int bj, int bk) {
  return o->ex[l][bidx(o, l, bi, bj, bk)] != 0;
}
static int block_is_leaf(const orc *o, int l, int bi, int bj, int bk) {
  if (!block_exists(o, l, bi, bj, bk)) return 0;
  if (l == o->L) return 1;
  return !block_exists(o, l + 1, 2 * bi, 2 * bj, o->dim == 3 ? 2 * bk : 0);
}
static int cell_block_exists(const orc *o, int l, int i, int j, int k) {
  return block_exists(o, l, i / OB, j / OB, k / OB);
}
static int cell_block_internal(const orc *o, int l, int i, int j, int k) {
  return cell_block_exists(o, l, i, j, k) && !block_is_leaf(o, l, i / OB, j / OB, k / OB);
}

/* ------------------------------------------------------------------------ */
/* equation of state (Section 2): p = (gamma-1) (rho e - rho |v|^2 / 2)       */

/* conservative (rho, rho v_1..rho v_d, rho e) -> primitive (rho, v_1..v_3, p) */
static void cons_to_prim(const orc *o, const double *Q, double *w) {
  double rho = Q[0];
  double v[3] = {0.0, 0.0, 0.0};
  for (int d = 0; d < o->dim; d++) v[d] = Q[1 + d] / rho;
  double vv = ((v[0] * v[0]) + (v[1] * v[1])) + (v[2] * v[2]);
  double E = Q[o->dim + 1];
  w[0] = rho;
  w[1] = v[0]; w[2] = v[1]; w[3] = v[2];
  w[4] = (o->gamma - 1.0) * (E - ((0.5 * rho) * vv));
}
static void prim_to_cons(const orc *o, const double *w, double *Q) {
  double vv = ((w[1] * w[1]) + (w[2] * w[2])) + (w[3] * w[3]);
  Q[0] = w[0];
  for (int d = 0; d < o->dim; d++) Q[1 + d] = w[0] * w[1 + d];
  Q[o->dim + 1] = (w[4] / (o->gamma - 1.0)) + ((0.5 * w[0]) * vv);
}

/* ------------------------------------------------------------------------ */
/* MUSCL reconstruction with the van Albada limiter (Section 2).
   Reading: primitive variables are reconstructed; the slope is
   a*b*(a+b)/(a^2+b^2) when a*b > 0 and 0 otherwise (no epsilon).  This slope
   never exceeds 1.21*min(|a|,|b|) in size, so w_i -/+ slope/2 stays positive
   whenever the three cells are positive and no first-order fallback is needed. */
static double van_albada(double a, double b) {
  double ab = a * b;
  if (ab > 0.0) return (ab * (a + b)) / ((a * a) + (b * b));
  return 0.0;
}

/* ------------------------------------------------------------------------ */
/* AUSM+ (Liou 1996, cited in Section 2).  Split Mach numbers and pressures with
   beta = 1/8, alpha = 3/16; interface sound speed = arithmetic mean (reading);
   |M| >= 1 takes the supersonic branch (both branches agree there). */
static double mach4_plus(double M) {
  if (fabs(M) >= 1.0) return 0.5 * (M + fabs(M));
  double t = M + 1.0, u = (M * M) - 1.0;
  return (0.25 * (t * t)) + (0.125 * (u * u));
}
static double mach4_minus(double M) {
  if (fabs(M) >= 1.0) return 0.5 * (M - fabs(M));
  double t = M - 1.0, u = (M * M) - 1.0;
  return (-0.25 * (t * t)) - (0.125 * (u * u));
}
static double pres5_plus(double M) {
  if (fabs(M) >= 1.0) return M > 0.0 ? 1.0 : 0.0;
  double t = M + 1.0, u = (M * M) - 1.0;
  return ((0.25 * (t * t)) * (2.0 - M)) + ((0.1875 * M) * (u * u));
}
static double pres5_minus(double M) {
  if (fabs(M) >= 1.0) return M < 0.0 ? 1.0 : 0.0;
  double t = M - 1.0, u = (M * M) - 1.0;
  return ((0.25 * (t * t)) * (2.0 + M)) - ((0.1875 * M) * (u * u));
}
/* flux across a face with normal dir nd from primitive face states wl | wr */
static void ausm_plus(const orc *o, int nd, const double *wl, const double *wr, double *F) {
  double g = o->gamma;
  double cl = sqrt((g * wl[4]) / wl[0]);
  double cr = sqrt((g * wr[4]) / wr[0]);
  double ch = 0.5 * (cl + cr);
  double ml = wl[1 + nd] / ch;
  double mr = wr[1 + nd] / ch;
  double m = mach4_plus(ml) + mach4_minus(mr);
  double ph = (pres5_plus(ml) * wl[4]) + (pres5_minus(mr) * wr[4]);
  double a = ch * m;
  const double *wu = (m >= 0.0) ? wl : wr;
  double vv = ((wu[1] * wu[1]) + (wu[2] * wu[2])) + (wu[3] * wu[3]);
  double rhoH = ((g / (g - 1.0)) * wu[4]) + ((0.5 * wu[0]) * vv);
  double fr = a * wu[0];
  F[0] = fr;
  for (int d = 0; d < o->dim; d++) {
    double f = fr * wu[1 + d];
    if (d == nd) f = f + ph;
    F[1 + d] = f;
  }
  F[o->dim + 1] = a * rhoH;
}

/* physical flux f_n(q) of Eq. 2.2, used only by the consistency check */
static void physical_flux(const orc *o, int nd, const double *Q, double *F) {
  double w[5];
  cons_to_prim(o, Q, w);
  double vn = w[1 + nd];
  F[0] = Q[0] * vn;
  for (int d = 0; d < o->dim; d++) F[1 + d] = Q[1 + d] * vn + (d == nd ? w[4] : 0.0);
  F[o->dim + 1] = (Q[o->dim + 1] + w[4]) * vn;
}

/* ------------------------------------------------------------------------ */
/* The AMR scheme of Section 2 (scheme 1): MUSCL-Hancock with the Minmod limiter
   in the primitive variables rho, v, p (Section 4.2) and the AUSMDV flux of
   Wada and Liou (1997).  The step is one stage: face states are advanced half
   a step with the exact flux before the numerical flux is taken, which makes
   the update second order in time like the midpoint rule.
   Reading (the paper says "unsplit" and "second order"): the cell's
   extrapolated states are all advanced by the same half-step increment
   dQ = sum_m (dt/2)/dx_m (f_m(Q^{-m}) - f_m(Q^{+m})) over every direction m,
   the unsplit MUSCL-Hancock predictor; a predictor that used only the face's
   own direction would be first order in time for oblique flow.  So the states
   of a face need the slopes of its two cells in every direction, i.e. the cells
   diagonally next to the face (the halo corners).
   Reading: AUSMDV without the entropy and shock fixes, K = 10 in the blend. */

static double minmod(double a, double b) {
  if ((a * b) > 0.0) return fabs(a) < fabs(b) ? a : b;
  return 0.0;
}

/* exact flux f_n of Eq. 2.2 at primitive state w with conservative state Q */
static void exact_flux_prim(const orc *o, int nd, const double *w, const double *Q, double *F) {
  double vn = w[1 + nd], p = w[4];
  F[0] = Q[0] * vn;
  for (int d = 0; d < o->dim; d++) {
    double f = Q[1 + d] * vn;
    if (d == nd) f = f + p;
    F[1 + d] = f;
  }
  F[o->dim + 1] = (Q[o->dim + 1] + p) * vn;
}

/* Hancock face state: cell primitive state w with Minmod slopes s[m][.] in every
   direction m; the extrapolated states w -/+ s[m]/2 give the half-step increment
   dQ = sum over m (in direction order) of h_m (f_m(Q^{-m}) - f_m(Q^{+m})),
   h_m = (dt/2)/dx_m; returns the primitive state of Q^{side,nd} + dQ
   (side = +1: the state on the cell's high face in direction nd, -1: low face). */
static void hancock_state(const orc *o, int l, const double *w, double s[3][5], double dt, int nd, int side,
                          double *wout) {
  double dQ[5] = {0, 0, 0, 0, 0};
  double Qf[5] = {0, 0, 0, 0, 0};
  for (int m = 0; m < o->dim; m++) {
    double wm[5], wp[5], Qm[5], Qp[5], Fm[5], Fp[5];
    for (int k = 0; k < 5; k++) {
      wm[k] = w[k] - (0.5 * s[m][k]);
      wp[k] = w[k] + (0.5 * s[m][k]);
    }
    prim_to_cons(o, wm, Qm);
    prim_to_cons(o, wp, Qp);
    exact_flux_prim(o, m, wm, Qm, Fm);
    exact_flux_prim(o, m, wp, Qp, Fp);
    double h = (0.5 * dt) / o->dx[l][m];
    for (int v = 0; v < o->nv; v++) {
      double inc = h * (Fm[v] - Fp[v]);
      dQ[v] = (m == 0) ? inc : dQ[v] + inc;
    }
    if (m == nd)
      for (int v = 0; v < o->nv; v++) Qf[v] = side > 0 ? Qp[v] : Qm[v];
  }
  double Qb[5];
  for (int v = 0; v < o->nv; v++) Qb[v] = Qf[v] + dQ[v];
  cons_to_prim(o, Qb, wout);
  if (o->dim == 2) wout[3] = 0.0;
}

/* AUSMDV flux across a face with normal nd from primitive face states wl | wr:
   c_m = max(c_L, c_R); pressure-weighted split velocities; split pressures;
   normal momentum flux blended between AUSMV and AUSMD by
   s = min(1, K |p_R - p_L| / min(p_L, p_R)) / 2; tangential momentum and
   enthalpy upwinded by the mass flux. */
static void ausmdv(const orc *o, int nd, const double *wl, const double *wr, double *F) {
  double g = o->gamma;
  double rl = wl[0], rr = wr[0], pl = wl[4], pr = wr[4];
  double ul = wl[1 + nd], ur = wr[1 + nd];
  double cl = sqrt((g * pl) / rl), cr = sqrt((g * pr) / rr);
  double cm = cl > cr ? cl : cr;
  double pol = pl / rl, por = pr / rr;
  double al = (2.0 * pol) / (pol + por), ar = (2.0 * por) / (pol + por);
  double upl = 0.5 * (ul + fabs(ul)), umr = 0.5 * (ur - fabs(ur));
  double ulp, urm, plp, prm;
  if (fabs(ul) <= cm) {
    double t = ul + cm;
    ulp = (al * (((t * t) / (4.0 * cm)) - upl)) + upl;
    plp = pl * (((t * t) * (2.0 - (ul / cm))) / (4.0 * (cm * cm)));
  } else {
    ulp = upl;
    plp = ul > 0.0 ? pl : 0.0;
  }
  if (fabs(ur) <= cm) {
    double t = ur - cm;
    urm = (ar * ((-((t * t) / (4.0 * cm))) - umr)) + umr;
    prm = pr * (((t * t) * (2.0 + (ur / cm))) / (4.0 * (cm * cm)));
  } else {
    urm = umr;
    prm = ur < 0.0 ? pr : 0.0;
  }
  double mdot = (ulp * rl) + (urm * rr);
  double am = fabs(mdot);
  double ph = plp + prm;
  double pmin = pl < pr ? pl : pr;
  double sw = 0.5 * fmin(1.0, (10.0 * fabs(pr - pl)) / pmin);
  double fv = (ulp * (rl * ul)) + (urm * (rr * ur));
  double fd = 0.5 * ((mdot * (ul + ur)) - (am * (ur - ul)));
  double fn = ((0.5 + sw) * fv) + ((0.5 - sw) * fd);
  F[0] = mdot;
  for (int d = 0; d < o->dim; d++) {
    if (d == nd) F[1 + d] = fn + ph;
    else F[1 + d] = 0.5 * ((mdot * (wl[1 + d] + wr[1 + d])) - (am * (wr[1 + d] - wl[1 + d])));
  }
  double vvl = ((wl[1] * wl[1]) + (wl[2] * wl[2])) + (wl[3] * wl[3]);
  double vvr = ((wr[1] * wr[1]) + (wr[2] * wr[2])) + (wr[3] * wr[3]);
  double hl = ((g / (g - 1.0)) * pol) + (0.5 * vvl), hr = ((g / (g - 1.0)) * por) + (0.5 * vvr);
  F[o->dim + 1] = 0.5 * ((mdot * (hl + hr)) - (am * (hr - hl)));
}

/* ------------------------------------------------------------------------ */
/* helpers on dense level arrays                                             */

static void get_cell(const orc *o, int l, const double *A, long c, double *Q) {
  for (int v = 0; v < o->nv; v++) Q[v] = A[(long)v * o->ncell[l] + c];
}
static double *alloc_level(const orc *o, int l) {
  double *a = (double *)malloc(sizeof(double) * (size_t)o->nv * (size_t)o->ncell[l]);
  for (long m = 0; m < (long)o->nv * o->ncell[l]; m++) a[m] = NAN;
  return a;
}

/* ------------------------------------------------------------------------ */
/* MR projection (Section 2.1): a parent cell average is the mean of its 2^d
   children, summed in lexicographic child order (x offset fastest).          */
static double project_cell(const orc *o, int lf, const double *F, int v, int i, int j, int k) {
  long nc = o->ncell[lf];
  double s = 0.0;
  int kz = (o->dim == 3) ? 2 : 1;
  int first = 1;
  for (int c = 0; c < kz; c++)
    for (int b = 0; b < 2; b++)
      for (int a = 0; a < 2; a++) {
        double x = F[(long)v * nc + cidx(o, lf, 2 * i + a, 2 * j + b, o->dim == 3 ? 2 * k + c : 0)];
        if (first) { s = x; first = 0; } else s = s + x;
      }
  return s * (o->dim == 3 ? 0.125 : 0.25);
}

/* restrict level l+1 onto the internal (refined) blocks of level l */
static void restrict_level(orc *o, int l, double **arr) {
  for (int bk = 0; bk < o->nb[l][2]; bk++)
    for (int bj = 0; bj < o->nb[l][1]; bj++)
      for (int bi = 0; bi < o->nb[l][0]; bi++) {
        if (!block_exists(o, l, bi, bj, bk) || block_is_leaf(o, l, bi, bj, bk)) continue;
        int kz = o->dim == 3 ? OB : 1;
        for (int kk = 0; kk < kz; kk++)
          for (int jj = 0; jj < OB; jj++)
            for (int ii = 0; ii < OB; ii++) {
              int i = bi * OB + ii, j = bj * OB + jj, k = (o->dim == 3) ? bk * OB + kk : 0;
              long c = cidx(o, l, i, j, k);
              for (int v = 0; v < o->nv; v++)
                arr[l][(long)v * o->ncell[l] + c] = project_cell(o, l + 1, arr[l + 1], v, i, j, k);
            }
      }
}
static void restrict_all(orc *o, double **arr) {
  for (int l = o->L - 1; l >= 0; l--) restrict_level(o, l, arr);
}

/* ------------------------------------------------------------------------ */
/* MR prediction, third order (Section 2.1): quadratic interpolation of cell
   averages, tensor product over directions.  In 1D the two children of coarse
   cell k are Q_k +/- (Q_{k-1} - Q_{k+1})/8 (+ for the even child).  In d
   dimensions the product of these operators adds the mixed differences of the
   coarse 3^d neighbourhood with weights 1/64 and 1/512.  Coarse neighbours
   outside the domain come from the same boundary rule.
   Evaluation order (also fixes rounding): Q_k, then the first-order terms in
   direction order, then the mixed pairs (12, 13, 23), then the triple term. */
static double coarse_at(const orc *o, int lc, const double *C, int v, int i, int j, int k) {
  i = bc_cell(o, lc, 0, i); j = bc_cell(o, lc, 1, j); k = bc_cell(o, lc, 2, k);
  return C[(long)v * o->ncell[lc] + cidx(o, lc, i, j, k)];
}
static double predict_cell(const orc *o, int lf, const double *C, int v, int I, int J, int K) {
  int lc = lf - 1;
  int ki = I >> 1, kj = J >> 1, kk = K >> 1;
  double si = (I & 1) ? -1.0 : 1.0, sj = (J & 1) ? -1.0 : 1.0, sk = (K & 1) ? -1.0 : 1.0;
  if (o->dim == 2) {
    double q = coarse_at(o, lc, C, v, ki, kj, 0);
    double d1 = coarse_at(o, lc, C, v, ki - 1, kj, 0) - coarse_at(o, lc, C, v, ki + 1, kj, 0);
    double d2 = coarse_at(o, lc, C, v, ki, kj - 1, 0) - coarse_at(o, lc, C, v, ki, kj + 1, 0);
    double d12 = ((coarse_at(o, lc, C, v, ki - 1, kj - 1, 0) - coarse_at(o, lc, C, v, ki + 1, kj - 1, 0))
                  - coarse_at(o, lc, C, v, ki - 1, kj + 1, 0)) + coarse_at(o, lc, C, v, ki + 1, kj + 1, 0);
    double r = q + (si * 0.125) * d1;
    r = r + (sj * 0.125) * d2;
    r = r + ((si * sj) * 0.015625) * d12;
    return r;
  }
  /* 3D */
  double q = coarse_at(o, lc, C, v, ki, kj, kk);
  double d1 = coarse_at(o, lc, C, v, ki - 1, kj, kk) - coarse_at(o, lc, C, v, ki + 1, kj, kk);
  double d2 = coarse_at(o, lc, C, v, ki, kj - 1, kk) - coarse_at(o, lc, C, v, ki, kj + 1, kk);
  double d3 = coarse_at(o, lc, C, v, ki, kj, kk - 1) - coarse_at(o, lc, C, v, ki, kj, kk + 1);
  double d12 = ((coarse_at(o, lc, C, v, ki - 1, kj - 1, kk) - coarse_at(o, lc, C, v, ki + 1, kj - 1, kk))
                - coarse_at(o, lc, C, v, ki - 1, kj + 1, kk)) + coarse_at(o, lc, C, v, ki + 1, kj + 1, kk);
  double d13 = ((coarse_at(o, lc, C, v, ki - 1, kj, kk - 1) - coarse_at(o, lc, C, v, ki + 1, kj, kk - 1))
                - coarse_at(o, lc, C, v, ki - 1, kj, kk + 1)) + coarse_at(o, lc, C, v, ki + 1, kj, kk + 1);
  double d23 = ((coarse_at(o, lc, C, v, ki, kj - 1, kk - 1) - coarse_at(o, lc, C, v, ki, kj + 1, kk - 1))
                - coarse_at(o, lc, C, v, ki, kj - 1, kk + 1)) + coarse_at(o, lc, C, v, ki, kj + 1, kk + 1);
  double e_lo = ((coarse_at(o, lc, C, v, ki - 1, kj - 1, kk - 1) - coarse_at(o, lc, C, v, ki + 1, kj - 1, kk - 1))
                 - coarse_at(o, lc, C, v, ki - 1, kj + 1, kk - 1)) + coarse_at(o, lc, C, v, ki + 1, kj + 1, kk - 1);
  double e_hi = ((coarse_at(o, lc, C, v, ki - 1, kj - 1, kk + 1) - coarse_at(o, lc, C, v, ki + 1, kj - 1, kk + 1))
                 - coarse_at(o, lc, C, v, ki - 1, kj + 1, kk + 1)) + coarse_at(o, lc, C, v, ki + 1, kj + 1, kk + 1);
  double d123 = e_lo - e_hi;
  double r = q + (si * 0.125) * d1;
  r = r + (sj * 0.125) * d2;
  r = r + (sk * 0.125) * d3;
  r = r + ((si * sj) * 0.015625) * d12;
  r = r + ((si * sk) * 0.015625) * d13;
  r = r + ((sj * sk) * 0.015625) * d23;
  r = r + (((si * sj) * sk) * 0.001953125) * d123;
  return r;
}

/* The same prediction in single precision: used to take the thresholding
   decision in the precision of a single-precision state. */
static float coarse_at_f(const orc *o, int lc, const float *C, int v, int i, int j, int k) {
  i = bc_cell(o, lc, 0, i); j = bc_cell(o, lc, 1, j); k = bc_cell(o, lc, 2, k);
  return C[(long)v * o->ncell[lc] + cidx(o, lc, i, j, k)];
}
static float predict_cell_f(const orc *o, int lf, const float *C, int v, int I, int J, int K) {
  int lc = lf - 1;
  int ki = I >> 1, kj = J >> 1, kk = K >> 1;
  float si = (I & 1) ? -1.0f : 1.0f, sj = (J & 1) ? -1.0f : 1.0f, sk = (K & 1) ? -1.0f : 1.0f;
  if (o->dim == 2) {
    float q = coarse_at_f(o, lc, C, v, ki, kj, 0);
    float d1 = coarse_at_f(o, lc, C, v, ki - 1, kj, 0) - coarse_at_f(o, lc, C, v, ki + 1, kj, 0);
    float d2 = coarse_at_f(o, lc, C, v, ki, kj - 1, 0) - coarse_at_f(o, lc, C, v, ki, kj + 1, 0);
    float d12 = ((coarse_at_f(o, lc, C, v, ki - 1, kj - 1, 0) - coarse_at_f(o, lc, C, v, ki + 1, kj - 1, 0))
                 - coarse_at_f(o, lc, C, v, ki - 1, kj + 1, 0)) + coarse_at_f(o, lc, C, v, ki + 1, kj + 1, 0);
    float r = q + (si * 0.125f) * d1;
    r = r + (sj * 0.125f) * d2;
    r = r + ((si * sj) * 0.015625f) * d12;
    return r;
  }
  float q = coarse_at_f(o, lc, C, v, ki, kj, kk);
  float d1 = coarse_at_f(o, lc, C, v, ki - 1, kj, kk) - coarse_at_f(o, lc, C, v, ki + 1, kj, kk);
  float d2 = coarse_at_f(o, lc, C, v, ki, kj - 1, kk) - coarse_at_f(o, lc, C, v, ki, kj + 1, kk);
  float d3 = coarse_at_f(o, lc, C, v, ki, kj, kk - 1) - coarse_at_f(o, lc, C, v, ki, kj, kk + 1);
  float d12 = ((coarse_at_f(o, lc, C, v, ki - 1, kj - 1, kk) - coarse_at_f(o, lc, C, v, ki + 1, kj - 1, kk))
               - coarse_at_f(o, lc, C, v, ki - 1, kj + 1, kk)) + coarse_at_f(o, lc, C, v, ki + 1, kj + 1, kk);
  float d13 = ((coarse_at_f(o, lc, C, v, ki - 1, kj, kk - 1) - coarse_at_f(o, lc, C, v, ki + 1, kj, kk - 1))
               - coarse_at_f(o, lc, C, v, ki - 1, kj, kk + 1)) + coarse_at_f(o, lc, C, v, ki + 1, kj, kk + 1);
  float d23 = ((coarse_at_f(o, lc, C, v, ki, kj - 1, kk - 1) - coarse_at_f(o, lc, C, v, ki, kj + 1, kk - 1))
               - coarse_at_f(o, lc, C, v, ki, kj - 1, kk + 1)) + coarse_at_f(o, lc, C, v, ki, kj + 1, kk + 1);
  float e_lo = ((coarse_at_f(o, lc, C, v, ki - 1, kj - 1, kk - 1) - coarse_at_f(o, lc, C, v, ki + 1, kj - 1, kk - 1))
                - coarse_at_f(o, lc, C, v, ki - 1, kj + 1, kk - 1)) + coarse_at_f(o, lc, C, v, ki + 1, kj + 1, kk - 1);
  float e_hi = ((coarse_at_f(o, lc, C, v, ki - 1, kj - 1, kk + 1) - coarse_at_f(o, lc, C, v, ki + 1, kj - 1, kk + 1))
                - coarse_at_f(o, lc, C, v, ki - 1, kj + 1, kk + 1)) + coarse_at_f(o, lc, C, v, ki + 1, kj + 1, kk + 1);
  float d123 = e_lo - e_hi;
  float r = q + (si * 0.125f) * d1;
  r = r + (sj * 0.125f) * d2;
  r = r + (sk * 0.125f) * d3;
  r = r + ((si * sj) * 0.015625f) * d12;
  r = r + ((si * sk) * 0.015625f) * d13;
  r = r + ((sj * sk) * 0.015625f) * d23;
  r = r + (((si * sj) * sk) * 0.001953125f) * d123;
  return r;
}

/* The level-l array the scheme sees: values of existing blocks from src, every
   other cell predicted from the level l-1 array coarse (virtual cells).  By
   gradedness every coarse value that a used virtual cell needs exists; absent
   coarse values are NaN and would poison any result that used them. */
static double *build_ext(const orc *o, int l, const double *src, const double *coarse) {
  double *e = alloc_level(o, l);
  /* every cell is written once from its own inputs (the pragma only matters in
     the OpenMP build of this file, used for the multi-core CPU baseline) */
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < o->n[l][2]; k++)
    for (int j = 0; j < o->n[l][1]; j++)
      for (int i = 0; i < o->n[l][0]; i++) {
        long c = cidx(o, l, i, j, k);
        if (cell_block_exists(o, l, i, j, k)) {
          for (int v = 0; v < o->nv; v++) e[(long)v * o->ncell[l] + c] = src[(long)v * o->ncell[l] + c];
        } else if (l > 0 && coarse) {
          for (int v = 0; v < o->nv; v++) e[(long)v * o->ncell[l] + c] = predict_cell(o, l, coarse, v, i, j, k);
        }
      }
  return e;
}

/* ------------------------------------------------------------------------ */
/* numerical flux across the face between cell a = (i,j,k) and a + e_nd,
   computed from the level array E (with boundary handling of indices); dt is
   the step the face states are advanced over (scheme 1 only) */
static void face_flux(const orc *o, int l, const double *E, int nd, int i, int j, int k, double dt, double *F) {
  int c4[4][3];
  for (int s = 0; s < 4; s++) {
    int p[3] = {i, j, k};
    p[nd] += s - 1; /* a-e, a, a+e, a+2e */
    for (int d = 0; d < 3; d++) c4[s][d] = bc_cell(o, l, d, p[d]);
  }
  double w[4][5];
  for (int s = 0; s < 4; s++) {
    double Q[5];
    get_cell(o, l, E, cidx(o, l, c4[s][0], c4[s][1], c4[s][2]), Q);
    cons_to_prim(o, Q, w[s]);
  }
  double wl[5], wr[5];
  if (o->scheme == O_SCHEME_HANCOCK) {
    /* the two cells of the face, their slopes in every direction */
    double sl[3][5], sr[3][5];
    for (int side = 0; side < 2; side++) {
      int c[3] = {i, j, k};
      c[nd] += side;
      double (*sp)[5] = side ? sr : sl;
      for (int m = 0; m < 3; m++)
        for (int q = 0; q < 5; q++) sp[m][q] = 0.0;
      for (int m = 0; m < o->dim; m++) {
        double wn[3][5];
        for (int t = 0; t < 3; t++) {
          int p[3] = {c[0], c[1], c[2]};
          p[m] += t - 1;
          double Q[5];
          get_cell(o, l, E, cidx(o, l, bc_cell(o, l, 0, p[0]), bc_cell(o, l, 1, p[1]), bc_cell(o, l, 2, p[2])), Q);
          cons_to_prim(o, Q, wn[t]);
        }
        for (int q = 0; q < 5; q++) {
          if (q >= 1 + o->dim && q < 4) continue;
          sp[m][q] = minmod(wn[1][q] - wn[0][q], wn[2][q] - wn[1][q]);
        }
      }
    }
    double wa[5], wb[5];
    for (int q = 0; q < 5; q++) { wa[q] = w[1][q]; wb[q] = w[2][q]; }
    if (o->dim == 2) { wa[3] = 0.0; wb[3] = 0.0; }
    hancock_state(o, l, wa, sl, dt, nd, +1, wl); /* high face of cell a */
    hancock_state(o, l, wb, sr, dt, nd, -1, wr); /* low face of cell a + e */
    ausmdv(o, nd, wl, wr, F);
    return;
  }
  for (int m = 0; m < 5; m++) {
    if (m >= 1 + o->dim && m < 4) { wl[m] = 0.0; wr[m] = 0.0; continue; }
    double sa = van_albada(w[1][m] - w[0][m], w[2][m] - w[1][m]);
    double sb = van_albada(w[2][m] - w[1][m], w[3][m] - w[2][m]);
    wl[m] = w[1][m] + 0.5 * sa;
    wr[m] = w[2][m] - 0.5 * sb;
  }
  ausm_plus(o, nd, wl, wr, F);
}

/* ------------------------------------------------------------------------ */
/* one RK stage on level l: out = q0 - coef*dt * F(E) on leaf blocks (or on all
   existing blocks when all_blocks), F = sum_n (F_{n,+} - F_{n,-}) / dx_n.
   When record is set, dt*F of both faces in every direction is stored per
   cell: coarse role overwritten, fine role written (first sub-step) or added. */
static void fv_level(orc *o, int l, const double *E, const double *q0, double *out,
                     double coef, double dt, int all_blocks, int record, int accumulate) {
  long nc = o->ncell[l];
  double lam[3];
  for (int d = 0; d < 3; d++) lam[d] = (coef * dt) / o->dx[l][d];
  /* blocks are independent: each cell's output and flux record is written once
     (the pragma only matters in the OpenMP build of this file) */
#pragma omp parallel for collapse(3) schedule(static)
  for (int bk = 0; bk < o->nb[l][2]; bk++)
    for (int bj = 0; bj < o->nb[l][1]; bj++)
      for (int bi = 0; bi < o->nb[l][0]; bi++) {
        if (all_blocks ? !block_exists(o, l, bi, bj, bk) : !block_is_leaf(o, l, bi, bj, bk)) continue;
        int kz = o->dim == 3 ? OB : 1;
        for (int kk = 0; kk < kz; kk++)
          for (int jj = 0; jj < OB; jj++)
            for (int ii = 0; ii < OB; ii++) {
              int i = bi * OB + ii, j = bj * OB + jj, k = (o->dim == 3) ? bk * OB + kk : 0;
              long c = cidx(o, l, i, j, k);
              double Fm[3][5], Fp[3][5];
              for (int d = 0; d < o->dim; d++) {
                int a[3] = {i, j, k};
                a[d] -= 1;
                face_flux(o, l, E, d, a[0], a[1], a[2], dt, Fm[d]);
                face_flux(o, l, E, d, i, j, k, dt, Fp[d]);
              }
              for (int v = 0; v < o->nv; v++) {
                double r = lam[0] * (Fp[0][v] - Fm[0][v]);
                r = r + lam[1] * (Fp[1][v] - Fm[1][v]);
                if (o->dim == 3) r = r + lam[2] * (Fp[2][v] - Fm[2][v]);
                out[(long)v * nc + c] = q0[(long)v * nc + c] - r;
              }
              if (record) {
                for (int d = 0; d < o->dim; d++)
                  for (int v = 0; v < o->nv; v++) {
                    long lo_i = ((long)(0 * 3 + d) * o->nv + v) * nc + c;
                    long hi_i = ((long)(1 * 3 + d) * o->nv + v) * nc + c;
                    double rm = dt * Fm[d][v], rp = dt * Fp[d][v];
                    o->rc[l][lo_i] = rm;
                    o->rc[l][hi_i] = rp;
                    if (accumulate) { o->rf[l][lo_i] = o->rf[l][lo_i] + rm; o->rf[l][hi_i] = o->rf[l][hi_i] + rp; }
                    else { o->rf[l][lo_i] = rm; o->rf[l][hi_i] = rp; }
                  }
              }
            }
      }
}

/* Flux correction (Section 2.2, Fig. 2; virtual leaves of Section 2.1): on every
   leaf cell of level l whose face borders a refined block of level l, the
   time-integrated coarse flux dt_l*F_c is replaced by the mean over the 2^{d-1}
   fine faces of the time-integrated fine fluxes (summed over the fine sub-steps):
   q += s * (R_c - mean R_f) / dx, s = +1 on the high face, -1 on the low face.
   The fine faces are averaged in lexicographic order of their tangential
   offsets (first tangential direction fastest). */
static void reflux_level(orc *o, int l, double *q) {
  if (l >= o->L) return;
  long nc = o->ncell[l], ncf = o->ncell[l + 1];
  for (int bk = 0; bk < o->nb[l][2]; bk++)
    for (int bj = 0; bj < o->nb[l][1]; bj++)
      for (int bi = 0; bi < o->nb[l][0]; bi++) {
        if (!block_is_leaf(o, l, bi, bj, bk)) continue;
        int kz = o->dim == 3 ? OB : 1;
        for (int kk = 0; kk < kz; kk++)
          for (int jj = 0; jj < OB; jj++)
            for (int ii = 0; ii < OB; ii++) {
              int i = bi * OB + ii, j = bj * OB + jj, k = (o->dim == 3) ? bk * OB + kk : 0;
              long c = cidx(o, l, i, j, k);
              for (int d = 0; d < o->dim; d++)
                for (int side = 0; side < 2; side++) {
                  int nbp[3] = {i, j, k};
                  nbp[d] += side ? 1 : -1;
                  /* neighbour cell across the face, with periodic wrap; none outside */
                  int ok = 1;
                  for (int e = 0; e < 3; e++) {
                    if (e >= o->dim) continue;
                    int N = o->n[l][e];
                    if (nbp[e] < 0 || nbp[e] >= N) {
                      if (o->bc == O_BC_PERIODIC) nbp[e] = (nbp[e] % N + N) % N; else ok = 0;
                    }
                  }
                  if (!ok || !cell_block_internal(o, l, nbp[0], nbp[1], nbp[2])) continue;
                  /* fine cells on the refined side adjacent to the face */
                  int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
                  double mean[5] = {0, 0, 0, 0, 0};
                  int nt2 = (o->dim == 3) ? 2 : 1;
                  int first = 1;
                  for (int b = 0; b < nt2; b++)
                    for (int a = 0; a < 2; a++) {
                      int f[3];
                      f[d] = side ? 2 * nbp[d] : 2 * nbp[d] + 1;
                      f[t1] = 2 * (t1 == 0 ? i : (t1 == 1 ? j : k)) + a;
                      if (o->dim == 3) f[t2] = 2 * (t2 == 1 ? j : k) + b; else f[2] = 0;
                      long fc = cidx(o, l + 1, f[0], f[1], f[2]);
                      int fside = side ? 0 : 1; /* the fine cell's face toward the coarse cell */
                      for (int v = 0; v < o->nv; v++) {
                        double x = o->rf[l + 1][((long)(fside * 3 + d) * o->nv + v) * ncf + fc];
                        if (first) mean[v] = x; else mean[v] = mean[v] + x;
                      }
                      first = 0;
                    }
                  for (int v = 0; v < o->nv; v++) {
                    double m = mean[v] * (o->dim == 3 ? 0.25 : 0.5);
                    double rcv = o->rc[l][((long)(side * 3 + d) * o->nv + v) * nc + c];
                    double corr = (rcv - m) / o->dx[l][d];
                    if (side) q[(long)v * nc + c] = q[(long)v * nc + c] + corr;
                    else q[(long)v * nc + c] = q[(long)v * nc + c] - corr;
                  }
                }
            }
      }
}

/* copy the cells of existing (or leaf-only) blocks of level l from src to dst */
static void copy_blocks(const orc *o, int l, const double *src, double *dst, int leaves_only) {
  long nc = o->ncell[l];
  for (int k = 0; k < o->n[l][2]; k++)
    for (int j = 0; j < o->n[l][1]; j++)
      for (int i = 0; i < o->n[l][0]; i++) {
        int keep = leaves_only ? block_is_leaf(o, l, i / OB, j / OB, k / OB) : cell_block_exists(o, l, i, j, k);
        if (!keep) continue;
        long c = cidx(o, l, i, j, k);
        for (int v = 0; v < o->nv; v++) dst[(long)v * nc + c] = src[(long)v * nc + c];
      }
}

/* ------------------------------------------------------------------------ */
/* creation, initial data                                                    */

orc *orc_create(int dim, int levels, const int *nb0, const double *lo, const double *hi,
                double gamma, int bc) {
  if (dim < 2 || dim > 3 || levels < 1 || levels > OMAXL) return NULL;
  orc *o = (orc *)calloc(1, sizeof(orc));
  o->dim = dim; o->nv = dim + 2; o->L = levels - 1; o->bc = bc; o->gamma = gamma;
  for (int d = 0; d < 3; d++) { o->lo[d] = lo[d]; o->hi[d] = hi[d]; }
  for (int l = 0; l <= o->L; l++) {
    o->ncell[l] = 1; o->nblk[l] = 1;
    for (int d = 0; d < 3; d++) {
      if (d < dim) { o->nb[l][d] = nb0[d] << l; o->n[l][d] = o->nb[l][d] * OB; }
      else { o->nb[l][d] = 1; o->n[l][d] = 1; }
      o->dx[l][d] = (d < dim) ? (hi[d] - lo[d]) / (double)o->n[l][d] : 1.0;
      o->ncell[l] *= o->n[l][d]; o->nblk[l] *= o->nb[l][d];
    }
    o->ex[l] = (uint8_t *)calloc((size_t)o->nblk[l], 1);
    o->sig[l] = (uint8_t *)calloc((size_t)o->nblk[l], 1);
    o->maxdet[l] = (double *)calloc((size_t)o->nblk[l], sizeof(double));
    o->q[l] = alloc_level(o, l);
    o->qs[l] = alloc_level(o, l);
    o->q0[l] = alloc_level(o, l);
    o->rc[l] = (double *)calloc((size_t)6 * o->nv * o->ncell[l], sizeof(double));
    o->rf[l] = (double *)calloc((size_t)6 * o->nv * o->ncell[l], sizeof(double));
  }
  return o;
}

/* threads the finite-volume loops use: 1, or the OpenMP team size in the
   OpenMP build of this file */
int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_destroy(orc *o) {
  if (!o) return;
  for (int l = 0; l <= o->L; l++) {
    free(o->ex[l]); free(o->sig[l]); free(o->maxdet[l]); free(o->q[l]); free(o->qs[l]);
    free(o->q0[l]); free(o->rc[l]); free(o->rf[l]);
  }
  free(o);
}

/* primitive initial state at a point */
static void ic_point(const orc *o, int kind, const double *P, const double *x, double *w) {
  w[0] = 1.0; w[1] = w[2] = w[3] = 0.0; w[4] = 1.0;
  if (kind == O_IC_QUADRANTS) {
    double xc = 0.5 * (o->lo[0] + o->hi[0]), yc = 0.5 * (o->lo[1] + o->hi[1]);
    int quad; /* I top-right, II top-left, III bottom-left, IV bottom-right (Table 1) */
    if (x[1] >= yc) quad = (x[0] >= xc) ? 0 : 1; else quad = (x[0] >= xc) ? 3 : 2;
    w[0] = P[4 * quad + 0]; w[1] = P[4 * quad + 1]; w[2] = P[4 * quad + 2]; w[4] = P[4 * quad + 3];
  } else if (kind == O_IC_ELLIPSOID) {
    double r2 = 0.0;
    for (int d = 0; d < 3; d++) { double t = (x[d] - P[d]) / P[3 + d]; r2 = r2 + t * t; }
    if (r2 < 1.0) { w[0] = P[6]; w[4] = P[7]; } else { w[0] = P[8]; w[4] = P[9]; }
  } else if (kind == O_IC_SHOCKTUBE) {
    int ax = (int)P[0];
    int left = x[ax] < P[1];
    w[0] = left ? P[2] : P[5];
    w[1 + ax] = left ? P[3] : P[6];
    w[4] = left ? P[4] : P[7];
  } else if (kind == O_IC_UNIFORM) {
    w[0] = P[0]; w[1] = P[1]; w[2] = P[2]; w[3] = P[3]; w[4] = P[4];
  } else if (kind == O_IC_WAVE) {
    double s = x[0] + x[1];
    if (o->dim == 3) s = s + x[2];
    w[0] = 1.0 + P[0] * sin(2.0 * M_PI * s);
    w[1] = P[1]; w[2] = P[2]; w[3] = P[3]; w[4] = P[4];
  } else if (kind == O_IC_ROTATED_ELLIPSOID) {
    double a = P[0], b = P[1], c = P[2], rc = P[3], th = P[4], ph = P[5];
    double x1 = x[0] * cos(th) - x[1] * sin(th);
    double t = x[0] * sin(th) + x[1] * cos(th);
    double x2 = t * cos(ph) - x[2] * sin(ph);
    double x3 = t * sin(ph) + x[2] * cos(ph);
    double r = sqrt((x1 / a) * (x1 / a) + (x2 / b) * (x2 / b) + (x3 / c) * (x3 / c));
    int in = r < rc;
    w[0] = in ? P[6] : P[8];
    w[4] = (o->gamma - 1.0) * (in ? P[7] : P[9]); /* at rest: p = (gamma-1) rho e */
  }
  if (o->dim == 2) w[3] = 0.0;
}

/* sample the finest level at cell centres (reading: no quadrature), project
   down to every coarser level; every block of every level exists */
int orc_init(orc *o, int kind, const double *P, int np) {
  (void)np;
  int L = o->L;
  for (int l = 0; l <= L; l++) memset(o->ex[l], 1, (size_t)o->nblk[l]);
  long nc = o->ncell[L];
  for (int k = 0; k < o->n[L][2]; k++)
    for (int j = 0; j < o->n[L][1]; j++)
      for (int i = 0; i < o->n[L][0]; i++) {
        double x[3] = {0.0, 0.0, 0.0};
        int id[3] = {i, j, k};
        for (int d = 0; d < o->dim; d++) x[d] = o->lo[d] + ((double)id[d] + 0.5) * o->dx[L][d];
        double w[5], Q[5];
        ic_point(o, kind, P, x, w);
        prim_to_cons(o, w, Q);
        long c = cidx(o, L, i, j, k);
        for (int v = 0; v < o->nv; v++) o->q[L][(long)v * nc + c] = Q[v];
      }
  restrict_all(o, o->q);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* dense access for the tests                                                */

long orc_level_cells(const orc *o, int l) { return o->ncell[l]; }
long orc_level_blocks(const orc *o, int l) { return o->nblk[l]; }
void orc_get_level(const orc *o, int l, double *out) {
  memcpy(out, o->q[l], sizeof(double) * (size_t)o->nv * (size_t)o->ncell[l]);
}
void orc_set_level(orc *o, int l, const double *in) {
  long nc = o->ncell[l];
  for (int k = 0; k < o->n[l][2]; k++)
    for (int j = 0; j < o->n[l][1]; j++)
      for (int i = 0; i < o->n[l][0]; i++) {
        long c = cidx(o, l, i, j, k);
        int e = cell_block_exists(o, l, i, j, k);
        for (int v = 0; v < o->nv; v++) o->q[l][(long)v * nc + c] = e ? in[(long)v * nc + c] : NAN;
      }
}
void orc_get_exist(const orc *o, int l, uint8_t *out) { memcpy(out, o->ex[l], (size_t)o->nblk[l]); }
/* replace the tree; cells of blocks that become absent turn NaN; cells of new
   blocks must be set by the caller (orc_set_level) */
void orc_set_exist(orc *o, int l, const uint8_t *in) {
  long nc = o->ncell[l];
  memcpy(o->ex[l], in, (size_t)o->nblk[l]);
  for (int k = 0; k < o->n[l][2]; k++)
    for (int j = 0; j < o->n[l][1]; j++)
      for (int i = 0; i < o->n[l][0]; i++)
        if (!cell_block_exists(o, l, i, j, k))
          for (int v = 0; v < o->nv; v++) o->q[l][(long)v * nc + cidx(o, l, i, j, k)] = NAN;
}
void orc_get_sig(const orc *o, int l, uint8_t *sig, double *maxdet) {
  memcpy(sig, o->sig[l], (size_t)o->nblk[l]);
  if (maxdet) memcpy(maxdet, o->maxdet[l], sizeof(double) * (size_t)o->nblk[l]);
}
void orc_get_scale(const orc *o, double *s) { for (int v = 0; v < o->nv; v++) s[v] = o->scale[v]; }
void orc_restrict_all(orc *o) { restrict_all(o, o->q); }

/* ------------------------------------------------------------------------ */
/* CFL time step (Section 2.2 "CFL-type condition"; readings: maximum over
   directions of |v_n| + c, minimum over the leaf cells).  With level-dependent
   steps the finest step is returned: each leaf's limit is scaled by 2^(l-L). */
double orc_dt(const orc *o, double cfl, int lts) {
  double best = INFINITY;
  for (int l = 0; l <= o->L; l++) {
    for (int k = 0; k < o->n[l][2]; k++)
      for (int j = 0; j < o->n[l][1]; j++)
        for (int i = 0; i < o->n[l][0]; i++) {
          if (!block_is_leaf(o, l, i / OB, j / OB, k / OB)) continue;
          double Q[5], w[5];
          get_cell(o, l, o->q[l], cidx(o, l, i, j, k), Q);
          cons_to_prim(o, Q, w);
          if (!(w[0] > 0.0) || !(w[4] > 0.0)) return -1.0;
          double c = sqrt((o->gamma * w[4]) / w[0]);
          for (int d = 0; d < o->dim; d++) {
            double r = o->dx[l][d] / (fabs(w[1 + d]) + c);
            if (lts) r = ldexp(r, l - o->L);
            if (r < best) best = r;
          }
        }
  }
  return cfl * best;
}

/* ------------------------------------------------------------------------ */
/* time stepping                                                             */

/* one step of explicit midpoint RK2 (Section 2) with one time step for all
   leaves: Q* = Q^n - dt/2 F(Q^n), Q^{n+1} = Q^n - dt F(Q*).  Virtual cells are
   predicted from the next coarser level of the same stage; refined blocks hold
   the projection of their children; the stage-2 fluxes at coarse-fine faces
   are corrected as in Fig. 2. */
static void step_global(orc *o, double dt) {
  int L = o->L;
  if (o->scheme == O_SCHEME_HANCOCK) {
    /* one MUSCL-Hancock stage from Q^n, fluxes recorded for the correction */
    double *qn[OMAXL];
    for (int l = 0; l <= L; l++) {
      qn[l] = alloc_level(o, l);
      double *E = build_ext(o, l, o->q[l], l > 0 ? o->q[l - 1] : NULL);
      fv_level(o, l, E, o->q[l], qn[l], 1.0, dt, 0, 1, 0);
      free(E);
    }
    for (int l = 0; l <= L; l++) {
      copy_blocks(o, l, qn[l], o->q[l], 1);
      free(qn[l]);
    }
    for (int l = 0; l < L; l++) reflux_level(o, l, o->q[l]);
    restrict_all(o, o->q);
    return;
  }
  /* stage 1 */
  for (int l = 0; l <= L; l++) {
    double *E = build_ext(o, l, o->q[l], l > 0 ? o->q[l - 1] : NULL);
    fv_level(o, l, E, o->q[l], o->qs[l], 0.5, dt, 0, 0, 0);
    free(E);
  }
  restrict_all(o, o->qs);
  /* stage 2 */
  double *qn[OMAXL];
  for (int l = 0; l <= L; l++) {
    qn[l] = alloc_level(o, l);
    double *E = build_ext(o, l, o->qs[l], l > 0 ? o->qs[l - 1] : NULL);
    fv_level(o, l, E, o->q[l], qn[l], 1.0, dt, 0, 1, 0);
    free(E);
  }
  for (int l = 0; l <= L; l++) {
    copy_blocks(o, l, qn[l], o->q[l], 1);
    free(qn[l]);
  }
  for (int l = 0; l < L; l++) reflux_level(o, l, o->q[l]);
  restrict_all(o, o->q);
}

/* q0 + theta*(q - q0) on existing blocks of level l (linear time interpolation) */
static double *time_interp(const orc *o, int l, double theta) {
  double *r = alloc_level(o, l);
  long nc = o->ncell[l];
  for (long m = 0; m < (long)o->nv * nc; m++) r[m] = o->q0[l][m] + theta * (o->q[l][m] - o->q0[l][m]);
  return r;
}

static int level_has_blocks(const orc *o, int l) {
  for (long b = 0; b < o->nblk[l]; b++) if (o->ex[l][b]) return 1;
  return 0;
}

/* Recursive level advance with level-dependent steps dt_l = 2^(L-l) dt_L
   (Section 2.1 MRLT, Section 2.2 Fig. 2): every existing block of level l is
   updated (refined ones are overwritten by the projection afterwards); virtual
   cells of level l are predicted from level l-1 interpolated linearly in time
   (stage 1 at the sub-step start, stage 2 at its midpoint); then level l+1 takes
   two sub-steps, is averaged onto level l, and the level-l leaves bordering it
   get the flux correction. */
static void advance_level(orc *o, int l, int sub, double dtL) {
  int L = o->L;
  /* Fig. 2: Remesh(l) before the update; at the first sub-step it would repeat
     the parent's Remesh(l-1), which regenerated these levels from the same data */
  if (o->lts_remesh && sub == 1 && l >= 1 && l < L) {
    if (o->rm_crit == O_CRIT_GRAD) remesh_amr(o, l, 0.5);
    else remesh_mr(o, l, 0.5);
  }
  double dtl = ldexp(dtL, L - l);
  double th1 = 0.5 * (double)sub, th2 = th1 + 0.25;
  copy_blocks(o, l, o->q[l], o->q0[l], 0);
  double *C1 = l > 0 ? time_interp(o, l - 1, th1) : NULL;
  double *E = build_ext(o, l, o->q[l], C1);
  double *qn = alloc_level(o, l);
  if (o->scheme == O_SCHEME_HANCOCK) {
    /* one stage from the sub-step start, ghosts at its start time */
    fv_level(o, l, E, o->q[l], qn, 1.0, dtl, 1, 1, sub == 1);
    free(E); free(C1);
  } else {
    fv_level(o, l, E, o->q[l], o->qs[l], 0.5, dtl, 1, 0, 0);
    free(E); free(C1);
    double *C2 = l > 0 ? time_interp(o, l - 1, th2) : NULL;
    E = build_ext(o, l, o->qs[l], C2);
    fv_level(o, l, E, o->q[l], qn, 1.0, dtl, 1, 1, sub == 1);
    free(E); free(C2);
  }
  copy_blocks(o, l, qn, o->q[l], 0);
  free(qn);
  if (l < L && level_has_blocks(o, l + 1)) {
    advance_level(o, l + 1, 0, dtL);
    advance_level(o, l + 1, 1, dtL);
    restrict_level(o, l, o->q);
    reflux_level(o, l, o->q[l]);
  }
}

/* one time step: global (lts = 0, dt for every leaf) or one coarse step of
   the level recursion (lts = 1, dt = finest-level step) */
void orc_step(orc *o, double dt, int lts) {
  o->rich_dt = dt; /* the step the Richardson estimate of the next flags takes */
  o->rich_lts = lts;
  if (lts) advance_level(o, 0, 0, dt);
  else step_global(o, dt);
}

/* ------------------------------------------------------------------------ */
/* MR analysis (Section 2.1): details d = Q_{l} - prediction from level l-1 on
   every existing block of level >= 1; a block is significant when
   max over cells and variables of |d_v| / s_v exceeds eps (strict), with the
   same eps on all levels.  Reading for the normalisation s_v (maxima over the
   level-0 field): s_rho = max|rho|, s_E = max|E|, s_m = max|rho| * max|v_n|,
   each at least 1e-14 * max|rho|.  precision 1: the state is rounded to single
   precision and the whole decision is taken in single precision. */
/* analysis of levels l0..L (significance of the others cleared); with th >= 0
   the details of level l0 are taken against the prediction from level l0-1
   interpolated in time (a remesh inside the level recursion) */
static int analyse_range(orc *o, double eps, int precision, long *n_sig, int l0, double th);
int orc_analyse(orc *o, double eps, int precision, long *n_sig) { return analyse_range(o, eps, precision, n_sig, 1, -1.0); }
static int analyse_range(orc *o, double eps, int precision, long *n_sig, int l0, double th) {
  int L = o->L, nv = o->nv, dim = o->dim;
  long total = 0;
  if (l0 < 1) l0 = 1;
  /* scales */
  double mr = 0.0, mE = 0.0, mv = 0.0;
  float fr = 0.0f, fE = 0.0f, fv = 0.0f;
  long nc0 = o->ncell[0];
  for (long c = 0; c < nc0; c++) {
    double rho = o->q[0][c], E = o->q[0][(long)(dim + 1) * nc0 + c];
    if (precision == 0) {
      if (fabs(rho) > mr) mr = fabs(rho);
      if (fabs(E) > mE) mE = fabs(E);
      for (int d = 0; d < dim; d++) {
        double v = fabs(o->q[0][(long)(1 + d) * nc0 + c] / rho);
        if (v > mv) mv = v;
      }
    } else {
      float rf = (float)rho, Ef = (float)E;
      if (fabsf(rf) > fr) fr = fabsf(rf);
      if (fabsf(Ef) > fE) fE = fabsf(Ef);
      for (int d = 0; d < dim; d++) {
        float v = fabsf((float)o->q[0][(long)(1 + d) * nc0 + c] / rf);
        if (v > fv) fv = v;
      }
    }
  }
  double s[5];
  float sf[5];
  if (precision == 0) {
    double fl = 1e-14 * mr;
    double sm = mr * mv;
    s[0] = mr > fl ? mr : fl;
    for (int d = 0; d < dim; d++) s[1 + d] = sm > fl ? sm : fl;
    s[dim + 1] = mE > fl ? mE : fl;
    for (int v = 0; v < nv; v++) o->scale[v] = s[v];
  } else {
    float fl = 1e-14f * fr;
    float sm = fr * fv;
    sf[0] = fr > fl ? fr : fl;
    for (int d = 0; d < dim; d++) sf[1 + d] = sm > fl ? sm : fl;
    sf[dim + 1] = fE > fl ? fE : fl;
    for (int v = 0; v < nv; v++) o->scale[v] = (double)sf[v];
  }
  memset(o->sig[0], 0, (size_t)o->nblk[0]);
  for (long b = 0; b < o->nblk[0]; b++) o->maxdet[0][b] = 0.0;
  float *qf[OMAXL] = {0};
  if (precision == 1)
    for (int l = 0; l <= L; l++) {
      qf[l] = (float *)malloc(sizeof(float) * (size_t)nv * (size_t)o->ncell[l]);
      for (long m = 0; m < (long)nv * o->ncell[l]; m++) qf[l][m] = (float)o->q[l][m];
    }
  for (int l = 1; l < l0 && l <= L; l++) {
    memset(o->sig[l], 0, (size_t)o->nblk[l]);
    for (long b = 0; b < o->nblk[l]; b++) o->maxdet[l][b] = 0.0;
  }
  for (int l = l0; l <= L; l++) {
    long nc = o->ncell[l];
    const double *P = o->q[l - 1];
    const float *Pf = precision == 1 ? qf[l - 1] : NULL;
    double *Pi = NULL;
    float *Pfi = NULL;
    if (l == l0 && th >= 0.0) {
      long n = (long)nv * o->ncell[l - 1];
      if (precision == 0) {
        Pi = time_interp(o, l - 1, th);
        P = Pi;
      } else {
        Pfi = (float *)malloc(sizeof(float) * (size_t)n);
        const float thf = (float)th;
        for (long m = 0; m < n; m++) {
          float a0 = (float)o->q0[l - 1][m];
          Pfi[m] = a0 + thf * ((float)o->q[l - 1][m] - a0);
        }
        Pf = Pfi;
      }
    }
    for (int bk = 0; bk < o->nb[l][2]; bk++)
      for (int bj = 0; bj < o->nb[l][1]; bj++)
        for (int bi = 0; bi < o->nb[l][0]; bi++) {
          long b = bidx(o, l, bi, bj, bk);
          o->sig[l][b] = 0;
          o->maxdet[l][b] = 0.0;
          if (!o->ex[l][b]) continue;
          double md = 0.0;
          float mdf = 0.0f;
          int kz = dim == 3 ? OB : 1;
          for (int kk = 0; kk < kz; kk++)
            for (int jj = 0; jj < OB; jj++)
              for (int ii = 0; ii < OB; ii++) {
                int i = bi * OB + ii, j = bj * OB + jj, k = (dim == 3) ? bk * OB + kk : 0;
                long c = cidx(o, l, i, j, k);
                for (int v = 0; v < nv; v++) {
                  if (precision == 0) {
                    double d = o->q[l][(long)v * nc + c] - predict_cell(o, l, P, v, i, j, k);
                    double r = fabs(d) / s[v];
                    if (r > md) md = r;
                  } else {
                    float d = qf[l][(long)v * nc + c] - predict_cell_f(o, l, Pf, v, i, j, k);
                    float r = fabsf(d) / sf[v];
                    if (r > mdf) mdf = r;
                  }
                }
              }
          if (precision == 0) { o->maxdet[l][b] = md; o->sig[l][b] = md > eps; }
          else { o->maxdet[l][b] = (double)mdf; o->sig[l][b] = mdf > (float)eps; }
          total += o->sig[l][b];
        }
    free(Pi);
    free(Pfi);
  }
  for (int l = 0; l <= L; l++) free(qf[l]);
  if (n_sig) *n_sig = total;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* scaled-gradient refinement flags with a one-cell buffer (Section 2.2):
   cell i is flagged when |rho(Q_{i+alpha}) - rho(Q_i)| > eps_w for some
   alpha in {0,1}^d \ {0} (reading: unscaled), or, with eps_p > 0 (the 3D case
   of Section 4.2 tests density and pressure), |p(Q_{i+alpha}) - p(Q_i)| > eps_p,
   p taken from the cell's conserved state (predicted from level l-1 where the
   cell's block is absent); a block of level
   l < L is flagged when a flagged cell lies within one cell of it.  Blocks are
   then grouped per row of the level's block grid into runs of at most 8 blocks
   (64 cells) whose flagged fraction stays >= eta_tol (reading of the
   clustering step); every block of a run is flagged for refinement. */
static double ext_pressure(const orc *o, int l, const double *E, long c) {
  double Q[5], w[5];
  get_cell(o, l, E, c, Q);
  cons_to_prim(o, Q, w);
  return w[4];
}
static int grad_flag_cell(const orc *o, int l, const double *E, int i, int j, int k, double epsw) {
  double r0 = E[cidx(o, l, i, j, k)];
  double p0 = o->eps_p > 0.0 ? ext_pressure(o, l, E, cidx(o, l, i, j, k)) : 0.0;
  int kz = o->dim == 3 ? 2 : 1;
  for (int c = 0; c < kz; c++)
    for (int b = 0; b < 2; b++)
      for (int a = 0; a < 2; a++) {
        if (a == 0 && b == 0 && c == 0) continue;
        int ii = bc_cell(o, l, 0, i + a), jj = bc_cell(o, l, 1, j + b), kk = bc_cell(o, l, 2, k + c);
        double r1 = E[cidx(o, l, ii, jj, kk)];
        if (fabs(r1 - r0) > epsw) return 1;
        if (o->eps_p > 0.0 && fabs(ext_pressure(o, l, E, cidx(o, l, ii, jj, kk)) - p0) > o->eps_p) return 1;
      }
  return 0;
}


/* ------------------------------------------------------------------------ */
/* Richardson estimate (Section 2.2: the heuristic local error indicator AMROC
   can add to the gradient flags; the estimate of Berger and Oliger 1984 and
   Berger and Colella 1989).  Reading (the paper gives no formula): with H_dt
   one step of the configured scheme over every cell of a uniform grid (the MR
   scheme: both stages of the midpoint rule; the AMR scheme: its one stage), R
   the mean of the 2^d children, E the level-l array the scheme sees and dt_l
   the step of level l in the last time step,
       tau = ( R H_dt(H_dt(E)) - H_2dt(R E) ) / (2^(o+1) - 2),   o = 2,
   on the level-l grid coarsened by 2, which keeps the boundary rule.  Only the
   density component is used. */

/* one stage over every cell of the grid of geometry slot gl:
   out = q0 - coef*dt * sum_n (F_{n,+} - F_{n,-}) / dx_n, directions in order */
static void grid_stage(const orc *o, int gl, const double *E, const double *q0, double *out, double coef,
                       double dt) {
  long nc = o->ncell[gl];
  double lam[3];
  for (int d = 0; d < 3; d++) lam[d] = (coef * dt) / o->dx[gl][d];
  for (int k = 0; k < o->n[gl][2]; k++)
    for (int j = 0; j < o->n[gl][1]; j++)
      for (int i = 0; i < o->n[gl][0]; i++) {
        long c = cidx(o, gl, i, j, k);
        double Fm[3][5], Fp[3][5];
        for (int d = 0; d < o->dim; d++) {
          int a[3] = {i, j, k};
          a[d] -= 1;
          face_flux(o, gl, E, d, a[0], a[1], a[2], dt, Fm[d]);
          face_flux(o, gl, E, d, i, j, k, dt, Fp[d]);
        }
        for (int v = 0; v < o->nv; v++) {
          double r = lam[0] * (Fp[0][v] - Fm[0][v]);
          r = r + lam[1] * (Fp[1][v] - Fm[1][v]);
          if (o->dim == 3) r = r + lam[2] * (Fp[2][v] - Fm[2][v]);
          out[(long)v * nc + c] = q0[(long)v * nc + c] - r;
        }
      }
}

/* H_dt on the grid of slot gl */
static void grid_scheme_step(const orc *o, int gl, const double *E, double *out, double dt) {
  if (o->scheme == O_SCHEME_HANCOCK) {
    grid_stage(o, gl, E, E, out, 1.0, dt);
    return;
  }
  double *S = alloc_level(o, gl);
  grid_stage(o, gl, E, E, S, 0.5, dt);
  grid_stage(o, gl, S, E, out, 1.0, dt);
  free(S);
}

/* tau (density) of level l on its grid coarsened by 2, which this sets up in the
   scratch geometry slot OG; tau has ncell[OG] entries */
static void rich_tau(orc *o, int l, const double *E, double dtl, double *tau) {
  o->ncell[OG] = 1;
  for (int d = 0; d < 3; d++) {
    o->n[OG][d] = d < o->dim ? o->n[l][d] / 2 : 1;
    o->nb[OG][d] = 0; /* no block structure */
    o->dx[OG][d] = d < o->dim ? 2.0 * o->dx[l][d] : 1.0;
    o->ncell[OG] *= o->n[OG][d];
  }
  long ncg = o->ncell[OG];
  double *F1 = alloc_level(o, l), *F2 = alloc_level(o, l);
  grid_scheme_step(o, l, E, F1, dtl);
  grid_scheme_step(o, l, F1, F2, dtl);
  double *RE = alloc_level(o, OG), *C1 = alloc_level(o, OG);
  for (int k = 0; k < o->n[OG][2]; k++)
    for (int j = 0; j < o->n[OG][1]; j++)
      for (int i = 0; i < o->n[OG][0]; i++)
        for (int v = 0; v < o->nv; v++) RE[(long)v * ncg + cidx(o, OG, i, j, k)] = project_cell(o, l, E, v, i, j, k);
  grid_scheme_step(o, OG, RE, C1, 2.0 * dtl);
  for (int k = 0; k < o->n[OG][2]; k++)
    for (int j = 0; j < o->n[OG][1]; j++)
      for (int i = 0; i < o->n[OG][0]; i++) {
        long c = cidx(o, OG, i, j, k);
        tau[c] = (project_cell(o, l, F2, 0, i, j, k) - C1[c]) / 6.0;
      }
  free(F1); free(F2); free(RE); free(C1);
}

/* coarse-cell flags |tau| > eps_r of the existing blocks of level l (OG set up by
   rich_tau), the largest |tau| of each block into maxdet[l].  The estimate of a
   block's coarse cells depends on E only within 8 fine cells of the block (two
   fine steps of at most two stages, each reaching 2 cells; one coarse step, 2
   coarse cells per stage); a block whose estimate is not finite, or whose E is
   not finite there, is counted (the limiters turn some absent, NaN, values
   into a zero slope, so the box is checked as well). */
static uint8_t *rich_flags(orc *o, int l, const double *E, double dtl) {
  long ncg = 1;
  for (int d = 0; d < o->dim; d++) ncg *= o->n[l][d] / 2;
  double *tau = (double *)malloc(sizeof(double) * (size_t)ncg);
  rich_tau(o, l, E, dtl, tau);
  uint8_t *rfl = (uint8_t *)calloc((size_t)ncg, 1);
  int kz = o->dim == 3 ? OB / 2 : 1;
  for (int bk = 0; bk < o->nb[l][2]; bk++)
    for (int bj = 0; bj < o->nb[l][1]; bj++)
      for (int bi = 0; bi < o->nb[l][0]; bi++) {
        long b = bidx(o, l, bi, bj, bk);
        if (!o->ex[l][b]) continue;
        int bad = 0;
        int z0 = o->dim == 3 ? bk * OB - OB : 0, z1 = o->dim == 3 ? bk * OB + 2 * OB : 1;
        for (int k = z0; k < z1; k++)
          for (int j = bj * OB - OB; j < bj * OB + 2 * OB; j++)
            for (int i = bi * OB - OB; i < bi * OB + 2 * OB; i++) {
              long c = cidx(o, l, bc_cell(o, l, 0, i), bc_cell(o, l, 1, j), bc_cell(o, l, 2, k));
              for (int v = 0; v < o->nv; v++)
                if (!isfinite(E[(long)v * o->ncell[l] + c])) bad = 1;
            }
        double m = 0.0;
        for (int c = 0; c < kz; c++)
          for (int bb = 0; bb < OB / 2; bb++)
            for (int a = 0; a < OB / 2; a++) {
              long q = cidx(o, OG, bi * (OB / 2) + a, bj * (OB / 2) + bb, o->dim == 3 ? bk * (OB / 2) + c : 0);
              double t = fabs(tau[q]);
              if (!isfinite(t)) bad = 1;
              if (t > o->eps_r) rfl[q] = 1;
              if (t > m) m = t;
            }
        o->maxdet[l][b] = m;
        o->rich_bad += bad;
      }
  free(tau);
  return rfl;
}

/* ------------------------------------------------------------------------ */
/* Berger-Rigoutsos clustering (Section 2.2, as in AMROC; Berger and Rigoutsos
   1991) of the flagged blocks fl of level l into boxes of blocks; every block of
   an accepted box is flagged for refinement in o->sig[l].  Reading on the block
   grid (the paper gives no details):
     - a box is first shrunk to the bounding box of its flagged blocks (dropped
       when it holds none);
     - it is accepted when flagged/volume >= eta and no side exceeds
       O_BR_MAX_SIDE blocks (64 cells, the largest patch side of the AMR
       workload);
     - an efficient box that is too long is bisected across its longest side;
     - otherwise it is cut at a hole (a slice with no flag) of the signatures
       (the counts of flags per slice along each direction): the first direction,
       in order, that has one, at the hole nearest the middle; else at the
       strongest inflection of the signatures (where the second difference
       changes sign, strength = the jump of the second difference), ties to the
       lower direction, then nearer the middle, then lower index; else the
       longest side (ties: lower direction) is bisected;
     - a cut at slice i gives [lo, i] and [i+1, hi]; both parts are clustered
       again. */
#define O_BR_MAX_SIDE 8
typedef struct { int lo[3], hi[3]; } obox;

static long br_flags_in(const orc *o, int l, const uint8_t *fl, const obox *b, obox *bb) {
  long cnt = 0;
  for (int d = 0; d < 3; d++) { bb->lo[d] = b->hi[d] + 1; bb->hi[d] = b->lo[d] - 1; }
  for (int k = b->lo[2]; k <= b->hi[2]; k++)
    for (int j = b->lo[1]; j <= b->hi[1]; j++)
      for (int i = b->lo[0]; i <= b->hi[0]; i++) {
        if (!fl[bidx(o, l, i, j, k)]) continue;
        int c[3] = {i, j, k};
        cnt++;
        for (int d = 0; d < 3; d++) {
          if (c[d] < bb->lo[d]) bb->lo[d] = c[d];
          if (c[d] > bb->hi[d]) bb->hi[d] = c[d];
        }
      }
  return cnt;
}

/* flags in slice s of box b along direction d */
static long br_slice(const orc *o, int l, const uint8_t *fl, const obox *b, int d, int s) {
  obox t = *b;
  t.lo[d] = s;
  t.hi[d] = s;
  long cnt = 0;
  for (int k = t.lo[2]; k <= t.hi[2]; k++)
    for (int j = t.lo[1]; j <= t.hi[1]; j++)
      for (int i = t.lo[0]; i <= t.hi[0]; i++) cnt += fl[bidx(o, l, i, j, k)] ? 1 : 0;
  return cnt;
}

static void br_box(orc *o, int l, const uint8_t *fl, obox b, double eta) {
  obox bb;
  long cnt = br_flags_in(o, l, fl, &b, &bb);
  if (cnt == 0) return;
  b = bb;
  long vol = 1;
  int longest = 0, big = 0;
  for (int d = 0; d < o->dim; d++) {
    int side = b.hi[d] - b.lo[d] + 1;
    vol *= side;
    if (side > O_BR_MAX_SIDE) big = 1;
    if (side > b.hi[longest] - b.lo[longest] + 1) longest = d;
  }
  int efficient = (double)cnt >= eta * (double)vol;
  if (efficient && !big) {
    for (int k = b.lo[2]; k <= b.hi[2]; k++)
      for (int j = b.lo[1]; j <= b.hi[1]; j++)
        for (int i = b.lo[0]; i <= b.hi[0]; i++) o->sig[l][bidx(o, l, i, j, k)] = 1;
    return;
  }
  int cd = -1, cut = 0;
  if (!efficient) {
    /* holes */
    for (int d = 0; d < o->dim && cd < 0; d++) {
      int best = -1;
      for (int s = b.lo[d] + 1; s < b.hi[d]; s++) {
        if (br_slice(o, l, fl, &b, d, s) != 0) continue;
        if (best < 0 || abs(2 * s - (b.lo[d] + b.hi[d])) < abs(2 * best - (b.lo[d] + b.hi[d]))) best = s;
      }
      if (best >= 0) { cd = d; cut = best; }
    }
    /* inflections */
    if (cd < 0) {
      long bstr = 0;
      for (int d = 0; d < o->dim; d++) {
        int n = b.hi[d] - b.lo[d] + 1;
        if (n < 4) continue;
        long *S = (long *)malloc(sizeof(long) * (size_t)n);
        for (int s = 0; s < n; s++) S[s] = br_slice(o, l, fl, &b, d, b.lo[d] + s);
        for (int s = 1; s + 2 < n; s++) {
          long l1 = S[s - 1] - 2 * S[s] + S[s + 1];
          long l2 = S[s] - 2 * S[s + 1] + S[s + 2];
          if (!((l1 < 0 && l2 > 0) || (l1 > 0 && l2 < 0))) continue;
          long str = labs(l2 - l1);
          int pos = b.lo[d] + s; /* cut between s and s + 1 */
          int better = 0;
          if (cd < 0 || str > bstr) better = 1;
          else if (str == bstr && d == cd) {
            int dm = abs(2 * pos + 1 - (b.lo[d] + b.hi[d])), cm = abs(2 * cut + 1 - (b.lo[d] + b.hi[d]));
            if (dm < cm) better = 1;
          }
          if (better) { cd = d; cut = pos; bstr = str; }
        }
        free(S);
      }
    }
  }
  if (cd < 0) {
    cd = longest;
    cut = (b.lo[cd] + b.hi[cd]) / 2;
  }
  obox a = b, c = b;
  a.hi[cd] = cut;
  c.lo[cd] = cut + 1;
  br_box(o, l, fl, a, eta);
  br_box(o, l, fl, c, eta);
}

static void br_cluster_level(orc *o, int l, const uint8_t *fl, double eta) {
  obox b;
  for (int d = 0; d < 3; d++) { b.lo[d] = 0; b.hi[d] = o->nb[l][d] - 1; }
  br_box(o, l, fl, b, eta);
}

/* flags of levels l0..L-1 (sig of every other level cleared); with th >= 0 the
   absent cells of level l0 are predicted from level l0-1 interpolated in time
   (th between its step's start and end), as its ghost cells are */
static void grad_flags_range(orc *o, double epsw, double eta, int l0, double th) {
  int L = o->L, dim = o->dim;
  for (int l = 0; l <= L; l++) {
    memset(o->sig[l], 0, (size_t)o->nblk[l]);
    memset(o->maxdet[l], 0, sizeof(double) * (size_t)o->nblk[l]);
  }
  for (int l = l0; l < L; l++) {
    double *C = NULL;
    if (l > 0) C = (l == l0 && th >= 0.0) ? time_interp(o, l - 1, th) : o->q[l - 1];
    double *E = build_ext(o, l, o->q[l], C);
    if (C && C != o->q[l - 1]) free(C);
    /* Richardson flags of level l (coarse cells of its grid coarsened by 2) */
    uint8_t *rfl = NULL;
    if (o->eps_r > 0.0) rfl = rich_flags(o, l, E, o->rich_lts ? ldexp(o->rich_dt, L - l) : o->rich_dt);
    uint8_t *fl = (uint8_t *)calloc((size_t)o->nblk[l], 1);
    for (int bk = 0; bk < o->nb[l][2]; bk++)
      for (int bj = 0; bj < o->nb[l][1]; bj++)
        for (int bi = 0; bi < o->nb[l][0]; bi++) {
          if (!block_exists(o, l, bi, bj, bk)) continue;
          int hit = 0;
          int k0 = dim == 3 ? bk * OB - 1 : 0, k1 = dim == 3 ? bk * OB + OB : 0;
          for (int k = k0; k <= k1 && !hit; k++)
            for (int j = bj * OB - 1; j <= bj * OB + OB && !hit; j++)
              for (int i = bi * OB - 1; i <= bi * OB + OB && !hit; i++) {
                int id[3] = {i, j, k}, ok = 1;
                for (int d = 0; d < dim; d++) {
                  if (id[d] < 0 || id[d] >= o->n[l][d]) {
                    if (o->bc == O_BC_PERIODIC) id[d] = bc_cell(o, l, d, id[d]); else ok = 0;
                  }
                }
                if (ok && grad_flag_cell(o, l, E, id[0], id[1], id[2], epsw)) hit = 1;
                if (ok && rfl && rfl[cidx(o, OG, id[0] >> 1, id[1] >> 1, id[2] >> 1)]) hit = 1;
              }
          fl[bidx(o, l, bi, bj, bk)] = (uint8_t)hit;
        }
    free(rfl);
    if (o->clustering == O_CLUSTER_BR) {
      br_cluster_level(o, l, fl, eta);
      free(fl);
      free(E);
      continue;
    }
    /* row clustering along the first direction */
    for (int bk = 0; bk < o->nb[l][2]; bk++)
      for (int bj = 0; bj < o->nb[l][1]; bj++) {
        int nx = o->nb[l][0];
        int x = 0;
        while (x < nx) {
          if (!fl[bidx(o, l, x, bj, bk)]) { x++; continue; }
          int best = x, cnt = 0;
          for (int e = x; e < nx && e - x < 8; e++) {
            if (fl[bidx(o, l, e, bj, bk)]) {
              cnt++;
              if ((double)cnt >= eta * (double)(e - x + 1)) best = e;
            }
          }
          for (int e = x; e <= best; e++) o->sig[l][bidx(o, l, e, bj, bk)] = 1;
          x = best + 1;
        }
      }
    free(fl);
    free(E);
  }
}
static void grad_flags(orc *o, double epsw, double eta) { grad_flags_range(o, epsw, eta, 0, -1.0); }

/* ------------------------------------------------------------------------ */
/* tree update (Section 2.1 refinement / coarsening, gradedness).  Block reading
   of the cell rules:
     MR:   a significant block B of level l >= 1 is kept, its 3^d-1 same-level
           neighbours are kept (safety zone), and for l < L its 2^d children are
           added (refinement by one level);
     GRAD: the children of every flagged block of level l < L are added;
   closure, level by level from the finest: a needed block brings its siblings
   (complete child sets), its parent, and the 3^d-1 neighbours of its parent
   (gradedness: at most one level between neighbouring leaves).  Blocks that
   leave the tree are dropped (the parent holds their projection); blocks that
   enter it are filled by the prediction from their parent level, coarse to
   fine.  Level 0 always exists. */
static void mark_nbrs(orc *o, uint8_t **need, int l, int bi, int bj, int bk) {
  int kz0 = o->dim == 3 ? -1 : 0, kz1 = o->dim == 3 ? 1 : 0;
  for (int c = kz0; c <= kz1; c++)
    for (int b = -1; b <= 1; b++)
      for (int a = -1; a <= 1; a++) {
        int x = bc_block(o, l, 0, bi + a), y = bc_block(o, l, 1, bj + b), z = bc_block(o, l, 2, bk + c);
        if (x < 0 || y < 0 || z < 0) continue;
        need[l][bidx(o, l, x, y, z)] = 1;
      }
}

int orc_adapt(orc *o, int crit, double eps, double epsw, double eta, int precision) {
  int L = o->L, dim = o->dim;
  if (crit == O_CRIT_MR) orc_analyse(o, eps, precision, NULL);
  else grad_flags(o, epsw, eta);
  uint8_t *need[OMAXL] = {0};
  for (int l = 0; l <= L; l++) need[l] = (uint8_t *)calloc((size_t)o->nblk[l], 1);
  memset(need[0], 1, (size_t)o->nblk[0]);
  for (int l = 0; l <= L; l++)
    for (int bk = 0; bk < o->nb[l][2]; bk++)
      for (int bj = 0; bj < o->nb[l][1]; bj++)
        for (int bi = 0; bi < o->nb[l][0]; bi++) {
          long b = bidx(o, l, bi, bj, bk);
          if (!o->ex[l][b] || !o->sig[l][b]) continue;
          if (crit == O_CRIT_MR) {
            if (l == 0) continue;
            need[l][b] = 1;
            mark_nbrs(o, need, l, bi, bj, bk);
          }
          if (l < L) {
            int kz = dim == 3 ? 2 : 1;
            for (int c = 0; c < kz; c++)
              for (int bb = 0; bb < 2; bb++)
                for (int a = 0; a < 2; a++)
                  need[l + 1][bidx(o, l + 1, 2 * bi + a, 2 * bj + bb, dim == 3 ? 2 * bk + c : 0)] = 1;
          }
        }
  for (int l = L; l >= 1; l--)
    for (int bk = 0; bk < o->nb[l][2]; bk++)
      for (int bj = 0; bj < o->nb[l][1]; bj++)
        for (int bi = 0; bi < o->nb[l][0]; bi++) {
          if (!need[l][bidx(o, l, bi, bj, bk)]) continue;
          int pi = bi >> 1, pj = bj >> 1, pk = bk >> 1;
          int kz = dim == 3 ? 2 : 1;
          for (int c = 0; c < kz; c++)
            for (int bb = 0; bb < 2; bb++)
              for (int a = 0; a < 2; a++)
                need[l][bidx(o, l, 2 * pi + a, 2 * pj + bb, dim == 3 ? 2 * pk + c : 0)] = 1;
          need[l - 1][bidx(o, l - 1, pi, pj, pk)] = 1;
          mark_nbrs(o, need, l - 1, pi, pj, pk);
        }
  apply_need(o, need, 1);
  for (int l = 0; l <= L; l++) free(need[l]);
  return 0;
}

/* Remesh(l0) of Fig. 2 (AMR with level-dependent steps): at the start of a
   sub-step of level l0, with every level >= l0 at the same time, the levels
   above l0 are regenerated from the gradient flags of levels l0..L-1 (level
   l0's absent cells predicted from level l0-1 interpolated in time, th); the
   tree of levels <= l0 is kept.  Reading of the nesting rule: the closure adds
   blocks above l0 only, and a block of level l0+1 or finer survives only where
   its parent and the parent's 3^d-1 neighbours are in the tree (finest last,
   so an unsupported block takes its descendants along). */
static void remesh_amr(orc *o, int l0, double th) {
  int L = o->L, dim = o->dim;
  grad_flags_range(o, o->rm_epsw, o->rm_eta, l0, th);
  uint8_t *need[OMAXL] = {0};
  for (int l = 0; l <= L; l++) {
    need[l] = (uint8_t *)calloc((size_t)o->nblk[l], 1);
    if (l <= l0) memcpy(need[l], o->ex[l], (size_t)o->nblk[l]);
  }
  int kz = dim == 3 ? 2 : 1;
  for (int l = l0; l < L; l++)
    for (int bk = 0; bk < o->nb[l][2]; bk++)
      for (int bj = 0; bj < o->nb[l][1]; bj++)
        for (int bi = 0; bi < o->nb[l][0]; bi++) {
          long b = bidx(o, l, bi, bj, bk);
          if (!o->ex[l][b] || !o->sig[l][b]) continue;
          for (int c = 0; c < kz; c++)
            for (int bb = 0; bb < 2; bb++)
              for (int a = 0; a < 2; a++)
                need[l + 1][bidx(o, l + 1, 2 * bi + a, 2 * bj + bb, dim == 3 ? 2 * bk + c : 0)] = 1;
        }
  close_and_nest(o, need, l0);
  apply_need(o, need, l0 + 1);
  for (int l = 0; l <= L; l++) free(need[l]);
}

/* closure above l0 (siblings; parents and their neighbours only above l0), then
   nesting: a block above l0 stays only where its parent and the parent's
   neighbours are needed (coarse to fine) */
static void close_and_nest(orc *o, uint8_t **need, int l0) {
  int L = o->L, dim = o->dim, kz = dim == 3 ? 2 : 1;
  for (int l = L; l > l0; l--)
    for (int bk = 0; bk < o->nb[l][2]; bk++)
      for (int bj = 0; bj < o->nb[l][1]; bj++)
        for (int bi = 0; bi < o->nb[l][0]; bi++) {
          if (!need[l][bidx(o, l, bi, bj, bk)]) continue;
          int pi = bi >> 1, pj = bj >> 1, pk = bk >> 1;
          for (int c = 0; c < kz; c++)
            for (int bb = 0; bb < 2; bb++)
              for (int a = 0; a < 2; a++)
                need[l][bidx(o, l, 2 * pi + a, 2 * pj + bb, dim == 3 ? 2 * pk + c : 0)] = 1;
          if (l - 1 > l0) {
            need[l - 1][bidx(o, l - 1, pi, pj, pk)] = 1;
            mark_nbrs(o, need, l - 1, pi, pj, pk);
          }
        }
  for (int l = l0 + 1; l <= L; l++)
    for (int bk = 0; bk < o->nb[l][2]; bk++)
      for (int bj = 0; bj < o->nb[l][1]; bj++)
        for (int bi = 0; bi < o->nb[l][0]; bi++) {
          long b = bidx(o, l, bi, bj, bk);
          if (!need[l][b]) continue;
          int pi = bi >> 1, pj = bj >> 1, pk = bk >> 1, ok = need[l - 1][bidx(o, l - 1, pi, pj, pk)] != 0;
          for (int c = (dim == 3 ? -1 : 0); c <= (dim == 3 ? 1 : 0) && ok; c++)
            for (int bb = -1; bb <= 1 && ok; bb++)
              for (int a = -1; a <= 1 && ok; a++) {
                int x = bc_block(o, l - 1, 0, pi + a), y = bc_block(o, l - 1, 1, pj + bb),
                    z = bc_block(o, l - 1, 2, pk + c);
                if (x < 0 || y < 0 || z < 0) continue;
                if (!need[l - 1][bidx(o, l - 1, x, y, z)]) ok = 0;
              }
          if (!ok) need[l][b] = 0;
        }
}

/* Remesh(l0) with the MR criterion, the same way as remesh_amr (the paper does
   not say when its MR code adapts inside the recursion; reading): details of
   levels l0..L from data at one time (level l0's against level l0-1
   interpolated in time, th); a significant block above l0 is kept with its
   neighbours and refined, a significant block of level l0 is refined; levels
   <= l0 are kept; closure and nesting above l0. */
static void remesh_mr(orc *o, int l0, double th) {
  int L = o->L, dim = o->dim, kz = dim == 3 ? 2 : 1;
  analyse_range(o, o->rm_eps, o->rm_precision, NULL, l0, th);
  uint8_t *need[OMAXL] = {0};
  for (int l = 0; l <= L; l++) {
    need[l] = (uint8_t *)calloc((size_t)o->nblk[l], 1);
    if (l <= l0) memcpy(need[l], o->ex[l], (size_t)o->nblk[l]);
  }
  for (int l = l0; l <= L; l++)
    for (int bk = 0; bk < o->nb[l][2]; bk++)
      for (int bj = 0; bj < o->nb[l][1]; bj++)
        for (int bi = 0; bi < o->nb[l][0]; bi++) {
          long b = bidx(o, l, bi, bj, bk);
          if (!o->ex[l][b] || !o->sig[l][b]) continue;
          if (l > l0) {
            need[l][b] = 1;
            mark_nbrs(o, need, l, bi, bj, bk);
          }
          if (l < L)
            for (int c = 0; c < kz; c++)
              for (int bb = 0; bb < 2; bb++)
                for (int a = 0; a < 2; a++)
                  need[l + 1][bidx(o, l + 1, 2 * bi + a, 2 * bj + bb, dim == 3 ? 2 * bk + c : 0)] = 1;
        }
  close_and_nest(o, need, l0);
  apply_need(o, need, l0 + 1);
  for (int l = 0; l <= L; l++) free(need[l]);
}

/* apply a needed-block map to levels lfrom..L, coarse to fine: drop, then
   predict new blocks from the level below */
static void apply_need(orc *o, uint8_t **need, int lfrom) {
  int L = o->L;
  for (int l = lfrom; l <= L; l++) {
    long nc = o->ncell[l];
    uint8_t *old = (uint8_t *)malloc((size_t)o->nblk[l]);
    memcpy(old, o->ex[l], (size_t)o->nblk[l]);
    memcpy(o->ex[l], need[l], (size_t)o->nblk[l]);
    for (int k = 0; k < o->n[l][2]; k++)
      for (int j = 0; j < o->n[l][1]; j++)
        for (int i = 0; i < o->n[l][0]; i++) {
          long b = bidx(o, l, i / OB, j / OB, k / OB), c = cidx(o, l, i, j, k);
          if (!need[l][b]) {
            for (int v = 0; v < o->nv; v++) o->q[l][(long)v * nc + c] = NAN;
          } else if (!old[b]) {
            for (int v = 0; v < o->nv; v++) o->q[l][(long)v * nc + c] = predict_cell(o, l, o->q[l - 1], v, i, j, k);
          }
        }
    free(old);
  }
}

/* ------------------------------------------------------------------------ */
/* diagnostics                                                               */

/* conserved totals: sum over leaf cells of Q_v times the cell volume */
void orc_totals(const orc *o, double *out) {
  for (int v = 0; v < o->nv; v++) out[v] = 0.0;
  for (int l = 0; l <= o->L; l++) {
    long nc = o->ncell[l];
    double vol = o->dx[l][0] * o->dx[l][1];
    if (o->dim == 3) vol = vol * o->dx[l][2];
    for (int k = 0; k < o->n[l][2]; k++)
      for (int j = 0; j < o->n[l][1]; j++)
        for (int i = 0; i < o->n[l][0]; i++) {
          if (!block_is_leaf(o, l, i / OB, j / OB, k / OB)) continue;
          long c = cidx(o, l, i, j, k);
          for (int v = 0; v < o->nv; v++) out[v] += o->q[l][(long)v * nc + c] * vol;
        }
  }
}

/* leaf representation projected to the finest level by repeated third-order
   prediction (Section 3, error assessment for MR) */
void orc_project_finest(const orc *o, double *out) {
  double *prev = NULL;
  for (int l = 0; l <= o->L; l++) {
    double *E = alloc_level(o, l);
    long nc = o->ncell[l];
    for (int k = 0; k < o->n[l][2]; k++)
      for (int j = 0; j < o->n[l][1]; j++)
        for (int i = 0; i < o->n[l][0]; i++) {
          long c = cidx(o, l, i, j, k);
          int ex = cell_block_exists(o, l, i, j, k);
          for (int v = 0; v < o->nv; v++)
            E[(long)v * nc + c] = ex ? o->q[l][(long)v * nc + c] : predict_cell(o, l, prev, v, i, j, k);
        }
    free(prev);
    prev = E;
  }
  memcpy(out, prev, sizeof(double) * (size_t)o->nv * (size_t)o->ncell[o->L]);
  free(prev);
}

/* AUSM+ flux of two conservative states (consistency checks) */
void orc_flux(orc *o, int nd, const double *Ql, const double *Qr, double *F) {
  double wl[5], wr[5];
  cons_to_prim(o, Ql, wl);
  cons_to_prim(o, Qr, wr);
  if (o->dim == 2) { wl[3] = 0.0; wr[3] = 0.0; }
  ausm_plus(o, nd, wl, wr, F);
}
void orc_physical_flux(orc *o, int nd, const double *Q, double *F) { physical_flux(o, nd, Q, F); }

/* AUSMDV flux of two conservative states (checks of the scheme-1 flux) */
void orc_flux_ausmdv(orc *o, int nd, const double *Ql, const double *Qr, double *F) {
  double wl[5], wr[5];
  cons_to_prim(o, Ql, wl);
  cons_to_prim(o, Qr, wr);
  if (o->dim == 2) { wl[3] = 0.0; wr[3] = 0.0; }
  ausmdv(o, nd, wl, wr, F);
}

/* Berger-Rigoutsos clustering of a given flag map of level l (tests of the
   clustering alone): out = the blocks of the accepted boxes */
void orc_br_cluster(orc *o, int l, const uint8_t *fl, double eta, uint8_t *out) {
  memset(o->sig[l], 0, (size_t)o->nblk[l]);
  br_cluster_level(o, l, fl, eta);
  memcpy(out, o->sig[l], (size_t)o->nblk[l]);
}

/* clustering of gradient flags: 0 = runs along the first direction, 1 = Berger-Rigoutsos */
int orc_set_clustering(orc *o, int mode) {
  if (mode != O_CLUSTER_ROWS && mode != O_CLUSTER_BR) return -1;
  o->clustering = mode;
  return 0;
}

/* Remesh(l) inside the level recursion (Fig. 2) for the gradient criterion
   with level-dependent steps: on with these flag parameters, or off */
int orc_set_lts_remesh(orc *o, int on, int crit, double eps, double epsw, double eta, int precision) {
  if ((on != 0 && on != 1) || (crit != O_CRIT_MR && crit != O_CRIT_GRAD) || (precision != 0 && precision != 1))
    return -1;
  o->lts_remesh = on;
  o->rm_crit = crit;
  o->rm_eps = eps;
  o->rm_epsw = epsw;
  o->rm_eta = eta;
  o->rm_precision = precision;
  return 0;
}

/* Richardson threshold added to the gradient criterion (0: off) */
int orc_set_eps_r(orc *o, double eps_r) {
  if (!(eps_r >= 0.0)) return -1;
  o->eps_r = eps_r;
  return 0;
}
long orc_rich_bad(const orc *o) { return o->rich_bad; }

/* Richardson estimate of density of level l with level step dt on the current
   state (absent cells predicted from level l-1): tau on the level's grid
   coarsened by 2 ([cell] layout, n_l/2 cells per dimension); returns the number
   of coarse cells of existing blocks whose estimate is not finite */
long orc_rich_tau(orc *o, int l, double dt, double *tau) {
  if (l < 0 || l > o->L) return -1;
  double *E = build_ext(o, l, o->q[l], l > 0 ? o->q[l - 1] : NULL);
  rich_tau(o, l, E, dt, tau);
  free(E);
  long bad = 0;
  int kz = o->dim == 3 ? o->n[OG][2] : 1;
  for (int k = 0; k < kz; k++)
    for (int j = 0; j < o->n[OG][1]; j++)
      for (int i = 0; i < o->n[OG][0]; i++)
        if (cell_block_exists(o, l, 2 * i, 2 * j, 2 * k) && !isfinite(tau[cidx(o, OG, i, j, k)])) bad++;
  return bad;
}

/* pressure threshold of the gradient criterion (0: density only) */
int orc_set_eps_p(orc *o, double eps_p) {
  if (!(eps_p >= 0.0)) return -1;
  o->eps_p = eps_p;
  return 0;
}

/* select the finite-volume scheme: 0 = MUSCL / van Albada / AUSM+ / RK2 midpoint
   (the MR scheme), 1 = MUSCL-Hancock / Minmod / AUSMDV (the AMR scheme) */
int orc_set_scheme(orc *o, int scheme) {
  if (scheme != O_SCHEME_MUSCL_RK2 && scheme != O_SCHEME_HANCOCK) return -1;
  o->scheme = scheme;
  return 0;
}

/* one cell's prediction from a given coarse level array (tests of the operator) */
double orc_predict(orc *o, int lf, const double *coarse, int v, int i, int j, int k) {
  return predict_cell(o, lf, coarse, v, i, j, k);
}
