/*
 * dispatch_oracle.c -- plain, slow FP64 CPU oracle of the per-patch update.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  It shares no code with
 * the CUDA path and must never be called by the product path.
 *
 * What it computes (DISPATCH I, Nordlund et al. 2018):
 *   - patches with guard zones on a periodic Cartesian level (Sec. 2.3,
 *     "cartesian" component; task/patch data types, Sec. 2.1), optionally
 *     with a second level at half the cell size: guard values across the
 *     resolution jump by conservative interpolation (prolongation) and
 *     averaging (restriction), Sec. 3 A;
 *   - a circular buffer of time slices per patch; a new state overwrites the
 *     oldest slice (Sec. 3 A, single-task view);
 *   - guard zones filled by linear interpolation in time from the neighbours'
 *     slices (Sec. 3 A and the closing paragraph of Sec. 3 B);
 *   - readiness by Eq. (1), t_self <= t_nbor + g dt_nbor, with grace g >= 0
 *     (guard values then extrapolated in time past a neighbour's newest
 *     slice), linear or quadratic time inter- and extrapolation (Sec. 3 B);
 *   - a dispatcher in two forms: a time-sorted ready queue (Sec. 3 B, mode i)
 *     and a sweep over the ready set (same schedule, see below);
 *   - local Courant time steps per patch (Sec. 5.1), quantised to powers of
 *     two so that patch times are exact dyadic numbers;
 *   - one step of ideal MHD per update.  The paper names its solvers (HLL-type
 *     Riemann solvers, Sec. 4.1; constrained transport with edge-centred
 *     electric fields, Sec. 4.3) but prints no scheme, so the scheme is the
 *     textbook one: primitive variables, MC-limited slopes, a MUSCL-Hancock
 *     half-step predictor, HLL face fluxes with Davis speed estimates, an
 *     upwind HLL edge EMF for constrained transport, and a conservative update.
 *
 * Every floating-point expression is written in a fixed evaluation order and
 * compiled with -ffp-contract=off, so that the result is a pure function of
 * the inputs.  No blocking or reordering: each stage loops over the whole
 * padded patch.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_EUNPHYS (-4)
#define ORC_EDEADLOCK (-6)
#define ORC_EBRACKET (-9)

enum { RHO = 0, VX = 1, VY = 2, VZ = 3, PR = 4, BX = 5, BY = 6, BZ = 7 };

/* Pressure floor of the primitive recovery, p >= PFLOOR * rho (a sound-speed
 * floor of 1e-10 in code units), as in the RAMSES solvers the paper ported
 * (Sec. 4.1).  The conserved energy is never modified. */
#define PFLOOR 1e-20

typedef struct {
  int level;  /* refinement level: 0, or 1 at half the cell size */
  int n[3];
  int64_t lo[3]; /* first interior cell in the level's index space */
  int nslot;
  double **U, **bx, **by, **bz; /* [slot] -> interior arrays */
  double *ts;                   /* time of each slot (NAN = empty) */
  double *smax;                 /* signal speed sum of each slot */
  int latest;
  double dt_last;
  int nnb;
  int *nb;
  int virt; /* 1: a copy of a patch another process owns (Sec. 3 C), never updated here */
} opatch;

typedef struct {
  int np;
  opatch *p;
  double gamma, cfl, t0, dt_max, dx; /* dx: level-0 cell size */
  int64_t L[2][3];                   /* cells per axis of the periodic box on each level */
  int nlev;                          /* 1, or 2 when level-1 patches exist */
  int g, nslot, time_mode, disp_mode;
  int riemann; /* face flux: 0 HLL, 1 HLLD */
  /* non-ideal MHD (Sec. 4.3): Ohmic resistivity eta, ambipolar drift
   * coefficient gamma_AD (gad) with ion density rho_i, and the Courant-like
   * factors of their step limits; a term is off when its coefficient is 0 */
  double eta, gad, rhoi, cohm, cad;
  /* grace g of Eq. 1 (0 <= g < 1) and the order of the time inter- and
   * extrapolation of guard values (1 linear, 2 quadratic), Sec. 3 B */
  double grace;
  int torder;
  int64_t nsched, capsched;
  int64_t *s_patch;
  double *s_t, *s_dt;
  int64_t n_updates, n_cells, n_sweeps, n_fallback;
  int64_t n_floor; /* cells of new slices whose pressure recovery took the floor */
  int nvirt;        /* virtual patches (Sec. 3 C); 0 in a whole-domain context */
  int status;
  char err[256];
} orc_ctx;

/* ------------------------------------------------------------------ */
/* Cell-level physics                                                  */
/* ------------------------------------------------------------------ */

/* Primitive state from conserved U = (rho, m, E) and the six faces of the
 * cell.  Heaviside-Lorentz units (E = -v x B, J = curl B, Sec. 4.3): total
 * energy E = p/(gamma-1) + rho v^2/2 + B^2/2; cell-centred B is the mean of
 * the two faces. */
static int prim(const double u[5], double bxl, double bxr, double byl, double byr,
                double bzl, double bzr, double gamma, double W[8]) {
  double rho = u[0];
  double irho = 1.0 / rho;
  double Bx = 0.5 * (bxl + bxr);
  double By = 0.5 * (byl + byr);
  double Bz = 0.5 * (bzl + bzr);
  double vx = u[1] * irho;
  double vy = u[2] * irho;
  double vz = u[3] * irho;
  double ke = 0.5 * rho * (vx * vx + vy * vy + vz * vz);
  double me = 0.5 * (Bx * Bx + By * By + Bz * Bz);
  double p = (gamma - 1.0) * (u[4] - ke - me);
  int floored = p < PFLOOR * rho;
  p = fmax(p, PFLOOR * rho);
  W[RHO] = rho; W[VX] = vx; W[VY] = vy; W[VZ] = vz; W[PR] = p;
  W[BX] = Bx; W[BY] = By; W[BZ] = Bz;
  return floored; /* 1 if the pressure floor was taken */
}

/* Fast magnetosonic speed along the axis whose field component is bn:
 * c_f^2 = [a^2 + B^2/rho + sqrt((a^2 + B^2/rho)^2 - 4 a^2 bn^2/rho)] / 2,
 * with irho = 1/rho. */
static double cfast(double gamma, double irho, double p, double bn, double bt1, double bt2) {
  double a2 = gamma * p * irho;
  double bb = (bn * bn + bt1 * bt1 + bt2 * bt2) * irho;
  double ca2 = bn * bn * irho;
  double s = a2 + bb;
  double disc = s * s - 4.0 * a2 * ca2;
  if (disc < 0.0) disc = 0.0;
  return sqrt(0.5 * (s + sqrt(disc)));
}

/* Monotonised-central limited slope: zero when the one-sided differences
 * have opposite signs or one of them is zero (a sign test, so no product is
 * formed that could underflow), else the smallest of twice either difference
 * and their mean, with their sign. */
static double mc(double dl, double dr) {
  if ((dl > 0.0 && dr < 0.0) || (dl < 0.0 && dr > 0.0) || dl == 0.0 || dr == 0.0) return 0.0;
  double s = fmin(fmin(2.0 * fabs(dl), 2.0 * fabs(dr)), 0.5 * fabs(dl + dr));
  return dl > 0.0 ? s : -s;
}

/* Hancock half-step predictor in primitive form, with d/dx_d replaced by the
 * limited slope dW_d (h = dt/(2 dx)):
 *   rho_t = -v.grad rho - rho div v
 *   v_t   = -(v.grad) v - (grad p + grad B^2/2 - (B.grad) B)/rho
 *   p_t   = -v.grad p - gamma p div v
 *   B_t   = (B.grad) v - (v.grad) B - B div v                              */
static void predict(const double W[8], const double *dX, const double *dY, const double *dZ,
                    double gamma, double h, double Ws[8]) {
  double rho = W[RHO], vx = W[VX], vy = W[VY], vz = W[VZ], p = W[PR];
  double Bx = W[BX], By = W[BY], Bz = W[BZ];
  double irho = 1.0 / rho;
  double divv = dX[VX] + dY[VY] + dZ[VZ];
  double r_rho = -(vx * dX[RHO] + vy * dY[RHO] + vz * dZ[RHO]) - rho * divv;
  double gpx = dX[PR] + (Bx * dX[BX] + By * dX[BY] + Bz * dX[BZ]);
  double gpy = dY[PR] + (Bx * dY[BX] + By * dY[BY] + Bz * dY[BZ]);
  double gpz = dZ[PR] + (Bx * dZ[BX] + By * dZ[BY] + Bz * dZ[BZ]);
  double tx = Bx * dX[BX] + By * dY[BX] + Bz * dZ[BX];
  double ty = Bx * dX[BY] + By * dY[BY] + Bz * dZ[BY];
  double tz = Bx * dX[BZ] + By * dY[BZ] + Bz * dZ[BZ];
  double r_vx = -(vx * dX[VX] + vy * dY[VX] + vz * dZ[VX]) - (gpx - tx) * irho;
  double r_vy = -(vx * dX[VY] + vy * dY[VY] + vz * dZ[VY]) - (gpy - ty) * irho;
  double r_vz = -(vx * dX[VZ] + vy * dY[VZ] + vz * dZ[VZ]) - (gpz - tz) * irho;
  double r_p = -(vx * dX[PR] + vy * dY[PR] + vz * dZ[PR]) - gamma * p * divv;
  double r_bx = (Bx * dX[VX] + By * dY[VX] + Bz * dZ[VX]) - (vx * dX[BX] + vy * dY[BX] + vz * dZ[BX]) - Bx * divv;
  double r_by = (Bx * dX[VY] + By * dY[VY] + Bz * dZ[VY]) - (vx * dX[BY] + vy * dY[BY] + vz * dZ[BY]) - By * divv;
  double r_bz = (Bx * dX[VZ] + By * dY[VZ] + Bz * dZ[VZ]) - (vx * dX[BZ] + vy * dY[BZ] + vz * dZ[BZ]) - Bz * divv;
  Ws[RHO] = rho + h * r_rho;
  Ws[VX] = vx + h * r_vx;
  Ws[VY] = vy + h * r_vy;
  Ws[VZ] = vz + h * r_vz;
  Ws[PR] = p + h * r_p;
  Ws[BX] = Bx + h * r_bx;
  Ws[BY] = By + h * r_by;
  Ws[BZ] = Bz + h * r_bz;
}

/* HLL flux through a face with normal axis d (Harten, Lax & van Leer 1983,
 * Davis speed estimates).  WL, WR are lab-frame primitive states; the normal
 * field of both is replaced by their mean.  Output F[0..4] in the lab frame
 * (mass, momentum x,y,z, energy), F[5], F[6] the induction fluxes of the two
 * tangential field components (cyclic order after d), S[0] = S_L, S[1] = S_R. */
static void hll(const double WL[8], const double WR[8], int d, double gamma, double F[7], double S[2]) {
  int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  double igm1 = 1.0 / (gamma - 1.0);
  double bn = 0.5 * (WL[BX + d] + WR[BX + d]);
  double FL[7], FR[7], UL[7], UR[7], cL, cR, vnL, vnR;
  for (int side = 0; side < 2; side++) {
    const double *W = side ? WR : WL;
    double *Fs = side ? FR : FL;
    double *Us = side ? UR : UL;
    double rho = W[RHO], p = W[PR];
    double vn = W[VX + d], vt1 = W[VX + t1], vt2 = W[VX + t2];
    double bt1 = W[BX + t1], bt2 = W[BX + t2];
    double v2 = vn * vn + vt1 * vt1 + vt2 * vt2;
    double B2 = bn * bn + bt1 * bt1 + bt2 * bt2;
    double E = p * igm1 + 0.5 * rho * v2 + 0.5 * B2;
    double PT = p + 0.5 * B2;
    double vB = vn * bn + vt1 * bt1 + vt2 * bt2;
    double cf = cfast(gamma, 1.0 / rho, p, bn, bt1, bt2);
    Us[0] = rho; Us[1] = rho * vn; Us[2] = rho * vt1; Us[3] = rho * vt2; Us[4] = E;
    Us[5] = bt1; Us[6] = bt2;
    Fs[0] = rho * vn;
    Fs[1] = rho * vn * vn + PT - bn * bn;
    Fs[2] = rho * vn * vt1 - bn * bt1;
    Fs[3] = rho * vn * vt2 - bn * bt2;
    Fs[4] = (E + PT) * vn - bn * vB;
    Fs[5] = vn * bt1 - vt1 * bn;
    Fs[6] = vn * bt2 - vt2 * bn;
    if (side) { cR = cf; vnR = vn; } else { cL = cf; vnL = vn; }
  }
  double SL = fmin(vnL - cL, vnR - cR);
  double SR = fmax(vnL + cL, vnR + cR);
  double Fr[7];
  double inv = 1.0 / (SR - SL);
  for (int c = 0; c < 7; c++) {
    if (SL >= 0.0) Fr[c] = FL[c];
    else if (SR <= 0.0) Fr[c] = FR[c];
    else Fr[c] = (SR * FL[c] - SL * FR[c] + SL * SR * (UR[c] - UL[c])) * inv;
  }
  F[0] = Fr[0];
  F[1 + d] = Fr[1];
  F[1 + t1] = Fr[2];
  F[1 + t2] = Fr[3];
  F[4] = Fr[4];
  F[5] = Fr[5];
  F[6] = Fr[6];
  S[0] = SL;
  S[1] = SR;
}

/* HLLD flux (Miyoshi & Kusano 2005) through a face with normal axis d: the
 * HLL outer speeds S_L, S_R (Davis estimates from the fast speeds, as in
 * hll), a contact at S_M with one total pressure pT* across the fan, two
 * rotational (Alfven) waves at S_M -+ |Bn|/sqrt(rho*), and the flux of the
 * region of the fan that holds x/t = 0.  Components as in hll (lab-frame
 * mass, momentum, energy, then the two tangential induction fluxes); S[0..1]
 * are S_L, S_R.  In the normal frame a state is (rho, u, v, w, p) with
 * tangential field (By, Bz) and the common normal field Bx.  Where
 * rho_a (S_a - u_a)(S_a - S_M) - Bx^2 vanishes (to 1e-12 of
 * rho_a (S_a - u_a)^2 + Bx^2) the star state keeps the tangential velocity
 * and field of its side. */
static void hlld_fan(const double WL[8], const double WR[8], int d, double gamma, double F[7], double S[2],
                     double *fan) {
  int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  double igm1 = 1.0 / (gamma - 1.0);
  double bx = 0.5 * (WL[BX + d] + WR[BX + d]);
  double rho[2], u[2], v[2], w[2], by[2], bz[2], E[2], PT[2], vB[2], c[2];
  double Fs[2][7], Us[2][7];
  for (int a = 0; a < 2; a++) {
    const double *W = a ? WR : WL;
    rho[a] = W[RHO]; u[a] = W[VX + d]; v[a] = W[VX + t1]; w[a] = W[VX + t2];
    by[a] = W[BX + t1]; bz[a] = W[BX + t2];
    double p = W[PR];
    double v2 = u[a] * u[a] + v[a] * v[a] + w[a] * w[a];
    double B2 = bx * bx + by[a] * by[a] + bz[a] * bz[a];
    E[a] = p * igm1 + 0.5 * rho[a] * v2 + 0.5 * B2;
    PT[a] = p + 0.5 * B2;
    vB[a] = u[a] * bx + v[a] * by[a] + w[a] * bz[a];
    c[a] = cfast(gamma, 1.0 / rho[a], p, bx, by[a], bz[a]);
    Us[a][0] = rho[a]; Us[a][1] = rho[a] * u[a]; Us[a][2] = rho[a] * v[a]; Us[a][3] = rho[a] * w[a];
    Us[a][4] = E[a]; Us[a][5] = by[a]; Us[a][6] = bz[a];
    Fs[a][0] = rho[a] * u[a];
    Fs[a][1] = rho[a] * u[a] * u[a] + PT[a] - bx * bx;
    Fs[a][2] = rho[a] * u[a] * v[a] - bx * by[a];
    Fs[a][3] = rho[a] * u[a] * w[a] - bx * bz[a];
    Fs[a][4] = (E[a] + PT[a]) * u[a] - bx * vB[a];
    Fs[a][5] = u[a] * by[a] - v[a] * bx;
    Fs[a][6] = u[a] * bz[a] - w[a] * bx;
  }
  double SL = fmin(u[0] - c[0], u[1] - c[1]);
  double SR = fmax(u[0] + c[0], u[1] + c[1]);
  double Fr[7];
  if (SL >= 0.0) {
    for (int k = 0; k < 7; k++) Fr[k] = Fs[0][k];
  } else if (SR <= 0.0) {
    for (int k = 0; k < 7; k++) Fr[k] = Fs[1][k];
  } else {
    double Sa[2] = {SL, SR};
    double dl = (SL - u[0]) * rho[0], dr = (SR - u[1]) * rho[1];
    double iden = 1.0 / (dr - dl);
    double SM = ((dr * u[1] - dl * u[0]) - PT[1] + PT[0]) * iden;
    double PTs = ((dr * PT[0] - dl * PT[1]) + dl * dr * (u[1] - u[0])) * iden;
    double rs[2], vs[2], ws[2], bys[2], bzs[2], Es[2], sr[2];
    for (int a = 0; a < 2; a++) {
      double su = Sa[a] - u[a];
      rs[a] = rho[a] * su / (Sa[a] - SM);
      double den = rho[a] * su * (Sa[a] - SM) - bx * bx;
      double ref = rho[a] * su * su + bx * bx;
      if (fabs(den) <= 1e-12 * ref) {
        vs[a] = v[a]; ws[a] = w[a]; bys[a] = by[a]; bzs[a] = bz[a];
      } else {
        double iv = 1.0 / den;
        double fv = bx * (SM - u[a]) * iv;
        double fb = (rho[a] * su * su - bx * bx) * iv;
        vs[a] = v[a] - by[a] * fv;
        ws[a] = w[a] - bz[a] * fv;
        bys[a] = by[a] * fb;
        bzs[a] = bz[a] * fb;
      }
      double vBs = SM * bx + vs[a] * bys[a] + ws[a] * bzs[a];
      Es[a] = ((su * E[a] - PT[a] * u[a] + PTs * SM) + bx * (vB[a] - vBs)) / (Sa[a] - SM);
      sr[a] = sqrt(rs[a]);
    }
    double aB = fabs(bx);
    double SsL = SM - aB / sr[0], SsR = SM + aB / sr[1];
    /* star states */
    double Ust[2][7];
    for (int a = 0; a < 2; a++) {
      Ust[a][0] = rs[a]; Ust[a][1] = rs[a] * SM; Ust[a][2] = rs[a] * vs[a]; Ust[a][3] = rs[a] * ws[a];
      Ust[a][4] = Es[a]; Ust[a][5] = bys[a]; Ust[a][6] = bzs[a];
    }
    /* double-star states (between the rotational waves) */
    double sg = bx > 0.0 ? 1.0 : bx < 0.0 ? -1.0 : 0.0;
    double isum = 1.0 / (sr[0] + sr[1]);
    double vss = ((sr[0] * vs[0] + sr[1] * vs[1]) + (bys[1] - bys[0]) * sg) * isum;
    double wss = ((sr[0] * ws[0] + sr[1] * ws[1]) + (bzs[1] - bzs[0]) * sg) * isum;
    double byss = ((sr[0] * bys[1] + sr[1] * bys[0]) + sr[0] * sr[1] * (vs[1] - vs[0]) * sg) * isum;
    double bzss = ((sr[0] * bzs[1] + sr[1] * bzs[0]) + sr[0] * sr[1] * (ws[1] - ws[0]) * sg) * isum;
    double vBss = SM * bx + vss * byss + wss * bzss;
    double Uss[2][7];
    for (int a = 0; a < 2; a++) {
      double vBsa = SM * bx + vs[a] * bys[a] + ws[a] * bzs[a];
      double Ess = a == 0 ? Es[0] - sr[0] * (vBsa - vBss) * sg : Es[1] + sr[1] * (vBsa - vBss) * sg;
      Uss[a][0] = rs[a]; Uss[a][1] = rs[a] * SM; Uss[a][2] = rs[a] * vss; Uss[a][3] = rs[a] * wss;
      Uss[a][4] = Ess; Uss[a][5] = byss; Uss[a][6] = bzss;
    }
    if (fan) {
      /* the whole fan, for checking: speeds S_L, S*_L, S_M, S*_R, S_R, the
       * normal-frame states U*_L, U**_L, U**_R, U*_R, and pT* */
      fan[0] = SL; fan[1] = SsL; fan[2] = SM; fan[3] = SsR; fan[4] = SR;
      fan[33] = PTs;
      for (int k = 0; k < 7; k++) {
        fan[5 + k] = Ust[0][k];
        fan[12 + k] = Uss[0][k];
        fan[19 + k] = Uss[1][k];
        fan[26 + k] = Ust[1][k];
      }
    }
    if (SsL >= 0.0) {
      for (int k = 0; k < 7; k++) Fr[k] = Fs[0][k] + SL * (Ust[0][k] - Us[0][k]);
    } else if (SsR <= 0.0) {
      for (int k = 0; k < 7; k++) Fr[k] = Fs[1][k] + SR * (Ust[1][k] - Us[1][k]);
    } else {
      int a = SM >= 0.0 ? 0 : 1;
      double Sst = a == 0 ? SsL : SsR;
      for (int k = 0; k < 7; k++)
        Fr[k] = ((Fs[a][k] + Sst * Uss[a][k]) - (Sst - Sa[a]) * Ust[a][k]) - Sa[a] * Us[a][k];
    }
  }
  F[0] = Fr[0];
  F[1 + d] = Fr[1];
  F[1 + t1] = Fr[2];
  F[1 + t2] = Fr[3];
  F[4] = Fr[4];
  F[5] = Fr[5];
  F[6] = Fr[6];
  S[0] = SL;
  S[1] = SR;
}

static void hlld(const double WL[8], const double WR[8], int d, double gamma, double F[7], double S[2]) {
  hlld_fan(WL, WR, d, gamma, F, S, NULL);
}

/* Upwind HLL edge EMF (two-dimensional HLL average of the four corner
 * states around an edge along axis e; a and b are the next two axes in cyclic
 * order).  Corner LL is the corner of the cell on the low side of both a and
 * b, RL the cell on the high-a/low-b side, LR low-a/high-b, RR high/high.
 * E_e at a corner is v_b B_a - v_a B_b (E = -v x B).  apa/ama are
 * max(0, +-S) over the two a-faces that touch the edge, apb/amb over the two
 * b-faces. */
static double emf(const double Wll[8], const double Wrl[8], const double Wlr[8], const double Wrr[8],
                  int e, double apa, double ama, double apb, double amb) {
  int a = (e + 1) % 3, b = (e + 2) % 3;
  double Ell = Wll[VX + b] * Wll[BX + a] - Wll[VX + a] * Wll[BX + b];
  double Erl = Wrl[VX + b] * Wrl[BX + a] - Wrl[VX + a] * Wrl[BX + b];
  double Elr = Wlr[VX + b] * Wlr[BX + a] - Wlr[VX + a] * Wlr[BX + b];
  double Err = Wrr[VX + b] * Wrr[BX + a] - Wrr[VX + a] * Wrr[BX + b];
  double BbL = 0.5 * (Wll[BX + b] + Wlr[BX + b]);
  double BbR = 0.5 * (Wrl[BX + b] + Wrr[BX + b]);
  double BaL = 0.5 * (Wll[BX + a] + Wrl[BX + a]);
  double BaR = 0.5 * (Wlr[BX + a] + Wrr[BX + a]);
  double num = apa * apb * Ell + ama * apb * Erl + apa * amb * Elr + ama * amb * Err;
  double den = (apa + ama) * (apb + amb);
  return num / den + apa * ama / (apa + ama) * (BbR - BbL) - apb * amb / (apb + amb) * (BaR - BaL);
}

/* Power of two not above x (x > 0), exact via frexp. */
static double pow2_floor(double x) {
  int e;
  frexp(x, &e);
  return ldexp(1.0, e - 1);
}

/* ------------------------------------------------------------------ */
/* Exported cell-level entry points (unit pins)                        */
/* ------------------------------------------------------------------ */
void orc_prim(const double *u, const double *faces, double gamma, double *W) {
  prim(u, faces[0], faces[1], faces[2], faces[3], faces[4], faces[5], gamma, W);
}
double orc_cfast(double gamma, double rho, double p, double bn, double bt1, double bt2) {
  return cfast(gamma, 1.0 / rho, p, bn, bt1, bt2);
}
double orc_mc(double dl, double dr) { return mc(dl, dr); }
void orc_predict(const double *W, const double *dX, const double *dY, const double *dZ, double gamma,
                 double h, double *Ws) {
  predict(W, dX, dY, dZ, gamma, h, Ws);
}
void orc_hll(const double *WL, const double *WR, int d, double gamma, double *F, double *S) {
  hll(WL, WR, d, gamma, F, S);
}
void orc_hlld(const double *WL, const double *WR, int d, double gamma, double *F, double *S) {
  hlld(WL, WR, d, gamma, F, S);
}
/* The HLLD fan (34 values, see hlld_fan) when S_L < 0 < S_R; returns 0 then,
 * 1 when the flux is a single side's. */
int orc_hlld_fan(const double *WL, const double *WR, int d, double gamma, double *fan) {
  double F[7], S[2];
  fan[0] = NAN;
  hlld_fan(WL, WR, d, gamma, F, S, fan);
  return isnan(fan[0]) ? 1 : 0;
}
double orc_emf(const double *Wll, const double *Wrl, const double *Wlr, const double *Wrr, int e,
               double apa, double ama, double apb, double amb) {
  return emf(Wll, Wrl, Wlr, Wrr, e, apa, ama, apb, amb);
}
double orc_pow2_floor(double x) { return pow2_floor(x); }

/* ------------------------------------------------------------------ */
/* Context, layout and neighbours                                      */
/* ------------------------------------------------------------------ */
static int64_t imod(int64_t a, int64_t m) {
  int64_t r = a % m;
  return r < 0 ? r + m : r;
}
static int64_t ncell(const opatch *P) { return (int64_t)P->n[0] * P->n[1] * P->n[2]; }
static int64_t nfx(const opatch *P) { return (int64_t)(P->n[0] + 1) * P->n[1] * P->n[2]; }
static int64_t nfy(const opatch *P) { return (int64_t)P->n[0] * (P->n[1] + 1) * P->n[2]; }
static int64_t nfz(const opatch *P) { return (int64_t)P->n[0] * P->n[1] * (P->n[2] + 1); }

/* Floor of a / b for b > 0. */
static int64_t fdiv(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

/* Does some periodic image of [qlo, qlo+qn) intersect [a, b)?  Writes the
 * set of intersecting image shifts as a bit mask (-L, 0, +L). */
static int ival_hit(int64_t a, int64_t b, int64_t qlo, int qn, int64_t L) {
  int mask = 0;
  for (int s = -1; s <= 1; s++) {
    int64_t qa = qlo + s * L, qb = qa + qn;
    if (qa < b && qb > a) mask |= 1 << (s + 1);
  }
  return mask;
}

/* The cells of the other level that patch P may read, along one axis, as a
 * half-open interval in that level's index space.  A level-1 patch reads
 * level-0 cells through prolongation: the parents of its padded cells and
 * one more coarse cell on each side (the limited slopes).  A level-0 patch
 * reads level-1 cells through restriction: the children of its padded cells
 * and of the cell above the top guard face. */
static void cross_interval(const opatch *P, int d, int g, int64_t *a, int64_t *b) {
  if (P->level == 1) {
    *a = fdiv(P->lo[d] - g, 2) - 1;
    *b = fdiv(P->lo[d] + P->n[d] + g - 1, 2) + 2;
  } else {
    *a = 2 * (P->lo[d] - g);
    *b = 2 * (P->lo[d] + P->n[d] + g) + 2;
  }
}

void orc_destroy(orc_ctx *c);

orc_ctx *orc_create(int np, const int32_t *n, const int64_t *lo, const int32_t *level, double gamma, double cfl,
                    double t0, double dt_max, const double *box_len, const int32_t *base, int nguard, int nslot,
                    int time_mode, int disp_mode) {
  if (np <= 0 || nguard < 2 || nslot < 3) return NULL;
  /* a patch must be wider than its guard depth so that every guard cell and
   * guard face lies in one of the adjacent patches */
  for (int i = 0; i < 3 * np; i++)
    if (n[i] <= nguard) return NULL;
  /* level-1 patches cover whole level-0 cells */
  for (int i = 0; i < np; i++) {
    int l = level ? level[i] : 0;
    if (l < 0 || l > 1) return NULL;
    if (l == 1)
      for (int d = 0; d < 3; d++)
        if ((n[3 * i + d] & 1) || (lo[3 * i + d] & 1)) return NULL;
  }
  orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
  c->np = np;
  c->gamma = gamma; c->cfl = cfl; c->t0 = t0; c->dt_max = dt_max;
  c->g = nguard; c->nslot = nslot; c->time_mode = time_mode; c->disp_mode = disp_mode;
  c->torder = 1;
  c->dx = box_len[0] / base[0];
  for (int d = 0; d < 3; d++) {
    c->L[0][d] = base[d];
    c->L[1][d] = 2 * (int64_t)base[d];
  }
  c->nlev = 1;
  c->p = (opatch *)calloc(np, sizeof(opatch));
  for (int i = 0; i < np; i++) {
    opatch *P = &c->p[i];
    P->level = level ? level[i] : 0;
    if (P->level == 1) c->nlev = 2;
    for (int d = 0; d < 3; d++) { P->n[d] = n[3 * i + d]; P->lo[d] = lo[3 * i + d]; }
    P->nslot = nslot;
    P->U = (double **)calloc(nslot, sizeof(double *));
    P->bx = (double **)calloc(nslot, sizeof(double *));
    P->by = (double **)calloc(nslot, sizeof(double *));
    P->bz = (double **)calloc(nslot, sizeof(double *));
    P->ts = (double *)malloc(nslot * sizeof(double));
    P->smax = (double *)calloc(nslot, sizeof(double));
    for (int s = 0; s < nslot; s++) {
      P->U[s] = (double *)calloc(5 * ncell(P), sizeof(double));
      P->bx[s] = (double *)calloc(nfx(P), sizeof(double));
      P->by[s] = (double *)calloc(nfy(P), sizeof(double));
      P->bz[s] = (double *)calloc(nfz(P), sizeof(double));
      P->ts[s] = NAN;
      if (!P->U[s] || !P->bx[s] || !P->by[s] || !P->bz[s]) { orc_destroy(c); return NULL; }
    }
    P->latest = 0;
    P->dt_last = 0.0;
  }
  /* neighbours.  Same level: every patch with an interior that some periodic
   * image puts inside this patch's padded box (the patch itself counts only
   * through a non-trivial image).  Other level: every patch whose interior
   * meets the cells this patch may read on that level (cross_interval), and,
   * so that the relation is symmetric, every patch that may read this one. */
  char *rel = (char *)calloc((size_t)np * np, 1);
  for (int i = 0; i < np; i++) {
    opatch *P = &c->p[i];
    for (int j = 0; j < np; j++) {
      opatch *Q = &c->p[j];
      int m[3], ok = 1;
      for (int d = 0; d < 3; d++) {
        int64_t a, b;
        if (Q->level == P->level) {
          a = P->lo[d] - nguard;
          b = P->lo[d] + P->n[d] + nguard;
        } else {
          cross_interval(P, d, nguard, &a, &b);
        }
        m[d] = ival_hit(a, b, Q->lo[d], Q->n[d], c->L[Q->level][d]);
        if (!m[d]) ok = 0;
      }
      if (!ok) continue;
      if (j == i && m[0] == 2 && m[1] == 2 && m[2] == 2) continue;
      rel[(size_t)i * np + j] = 1;
      rel[(size_t)j * np + i] = 1;
    }
  }
  int *tmp = (int *)malloc(sizeof(int) * np);
  for (int i = 0; i < np; i++) {
    opatch *P = &c->p[i];
    int cnt = 0;
    for (int j = 0; j < np; j++)
      if (rel[(size_t)i * np + j]) tmp[cnt++] = j;
    P->nnb = cnt;
    P->nb = (int *)malloc(sizeof(int) * (cnt > 0 ? cnt : 1));
    memcpy(P->nb, tmp, sizeof(int) * cnt);
  }
  free(tmp);
  free(rel);
  return c;
}

void orc_destroy(orc_ctx *c) {
  if (!c) return;
  for (int i = 0; i < c->np; i++) {
    opatch *P = &c->p[i];
    for (int s = 0; s < c->nslot; s++) {
      if (P->U) free(P->U[s]);
      if (P->bx) free(P->bx[s]);
      if (P->by) free(P->by[s]);
      if (P->bz) free(P->bz[s]);
    }
    free(P->U); free(P->bx); free(P->by); free(P->bz);
    free(P->ts); free(P->smax); free(P->nb);
  }
  free(c->p);
  free(c->s_patch); free(c->s_t); free(c->s_dt);
  free(c);
}

/* Face flux of every later update: 0 HLL (the default), 1 HLLD. */
int orc_set_riemann(orc_ctx *c, int riemann) {
  if (riemann != 0 && riemann != 1) return ORC_EINVAL;
  c->riemann = riemann;
  return ORC_OK;
}

/* Grace g of Eq. 1 (0 <= g < 1) and the order of the time inter- and
 * extrapolation of guard values (1 linear, 2 quadratic; Sec. 3 B).  g > 0
 * is taken with the sweep dispatcher only (a sweep updates every ready
 * patch from the slices before it, so the result does not depend on the
 * order of updates), and quadratic extrapolation (g > 0, order 2) needs
 * four slices so that the oldest patch can always step. */
int orc_set_time(orc_ctx *c, double grace, int order) {
  if (!(grace >= 0.0) || !(grace < 1.0) || (order != 1 && order != 2)) return ORC_EINVAL;
  if (grace > 0.0 && c->time_mode == 1 && c->disp_mode == 0) return ORC_EINVAL;
  if (grace > 0.0 && order == 2 && c->nslot < 4) return ORC_EINVAL;
  c->grace = grace;
  c->torder = order;
  return ORC_OK;
}

/* Non-ideal terms of every later update (Sec. 4.3): E_Ohm = eta J (Eq. 2)
 * and E_AD = -v_D x B with v_D = J x B / (gamma_AD rho rho_i) (Eqs. 5-6),
 * step limits C_Ohm dx^2 / eta (Eq. 4) and C_AD gamma_AD rho_i rho dx^2 / B^2
 * (Eq. 8).  eta = 0 or gamma_AD = 0 turns that term off. */
int orc_set_nonideal(orc_ctx *c, double eta, double gamma_ad, double rho_i, double c_ohm, double c_ad) {
  if (!(eta >= 0.0) || !(gamma_ad >= 0.0) || !(c_ohm > 0.0) || !(c_ad > 0.0)) return ORC_EINVAL;
  if (gamma_ad > 0.0 && !(rho_i > 0.0)) return ORC_EINVAL;
  c->eta = eta; c->gad = gamma_ad; c->rhoi = rho_i; c->cohm = c_ohm; c->cad = c_ad;
  return ORC_OK;
}

/* The diffusive step limits as a signal speed: dt = cfl dx / s equals
 * C_Ohm dx^2 / eta for s = cfl eta / (C_Ohm dx), and C_AD gamma_AD rho_i rho
 * dx^2 / B^2 for s = cfl B^2 / (C_AD gamma_AD rho_i rho dx); the larger of the
 * two (0 with both terms off).  W: primitive cell state, dxl: cell size. */
static double nonideal_speed(const orc_ctx *c, const double W[8], double dxl) {
  double s = 0.0;
  if (c->eta > 0.0) s = c->cfl * c->eta / (c->cohm * dxl);
  if (c->gad > 0.0) {
    double B2 = W[BX] * W[BX] + W[BY] * W[BY] + W[BZ] * W[BZ];
    double sad = c->cfl * B2 / ((((c->cad * c->gad) * c->rhoi) * W[RHO]) * dxl);
    s = fmax(s, sad);
  }
  return s;
}

int orc_num_nbors(orc_ctx *c, int P, int *out) {
  if (out) memcpy(out, c->p[P].nb, sizeof(int) * c->p[P].nnb);
  return c->p[P].nnb;
}

const char *orc_last_error(orc_ctx *c) { return c->err; }

/* Signal speed sum of a stored slice: max over interior cells of
 * sum_d (|v_d| + c_f,d). */
static double slice_smax(orc_ctx *c, opatch *P, int s, int *bad) {
  int nx = P->n[0], ny = P->n[1], nz = P->n[2];
  int64_t nc = ncell(P);
  double m = 0.0;
  *bad = 0;
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        int64_t id = ((int64_t)k * ny + j) * nx + i;
        double u[5], W[8];
        for (int q = 0; q < 5; q++) u[q] = P->U[s][q * nc + id];
        double bxl = P->bx[s][((int64_t)k * ny + j) * (nx + 1) + i];
        double bxr = P->bx[s][((int64_t)k * ny + j) * (nx + 1) + i + 1];
        double byl = P->by[s][((int64_t)k * (ny + 1) + j) * nx + i];
        double byr = P->by[s][((int64_t)k * (ny + 1) + j + 1) * nx + i];
        double bzl = P->bz[s][((int64_t)k * ny + j) * nx + i];
        double bzr = P->bz[s][((int64_t)(k + 1) * ny + j) * nx + i];
        prim(u, bxl, bxr, byl, byr, bzl, bzr, c->gamma, W);
        if (!(W[RHO] > 0.0) || !(W[PR] > 0.0)) *bad = 1;
        double ir = 1.0 / W[RHO];
        double cx = cfast(c->gamma, ir, W[PR], W[BX], W[BY], W[BZ]);
        double cy = cfast(c->gamma, ir, W[PR], W[BY], W[BZ], W[BX]);
        double cz = cfast(c->gamma, ir, W[PR], W[BZ], W[BX], W[BY]);
        double sum = (fabs(W[VX]) + cx) + (fabs(W[VY]) + cy) + (fabs(W[VZ]) + cz);
        sum = fmax(sum, nonideal_speed(c, W, ldexp(c->dx, -P->level)));
        if (sum > m) m = sum;
      }
  return m;
}

/* Load the initial state of every patch (concatenated in patch order, each
 * interior-only: U[5][nz][ny][nx], bx[nz][ny][nx+1], by[nz][ny+1][nx],
 * bz[nz+1][ny][nx]) into slot 0 at time t0. */
int orc_set_state(orc_ctx *c, const double *U, const double *bx, const double *by, const double *bz) {
  int64_t oU = 0, ox = 0, oy = 0, oz = 0;
  for (int i = 0; i < c->np; i++) {
    opatch *P = &c->p[i];
    for (int s = 0; s < c->nslot; s++) P->ts[s] = NAN;
    P->latest = 0;
    P->ts[0] = c->t0;
    P->dt_last = 0.0;
    memcpy(P->U[0], U + oU, sizeof(double) * 5 * ncell(P));
    memcpy(P->bx[0], bx + ox, sizeof(double) * nfx(P));
    memcpy(P->by[0], by + oy, sizeof(double) * nfy(P));
    memcpy(P->bz[0], bz + oz, sizeof(double) * nfz(P));
    oU += 5 * ncell(P); ox += nfx(P); oy += nfy(P); oz += nfz(P);
    int bad;
    P->smax[0] = slice_smax(c, P, 0, &bad);
    if (bad) { snprintf(c->err, sizeof c->err, "non-positive rho or p in patch %d", i); return ORC_EUNPHYS; }
  }
  c->nsched = 0;
  c->n_updates = c->n_cells = c->n_sweeps = c->n_fallback = c->n_floor = 0;
  c->status = 0;
  return ORC_OK;
}

/* Load one stored slot of one patch (used to reproduce a single update from
 * a saved dispatcher state).  The signal speed of the slot is recomputed. */
int orc_set_slot(orc_ctx *c, int ip, int s, double t, const double *U, const double *bx, const double *by,
                 const double *bz) {
  opatch *P = &c->p[ip];
  if (s < 0 || s >= c->nslot) return ORC_EINVAL;
  P->ts[s] = t;
  if (isnan(t)) return ORC_OK;
  memcpy(P->U[s], U, sizeof(double) * 5 * ncell(P));
  memcpy(P->bx[s], bx, sizeof(double) * nfx(P));
  memcpy(P->by[s], by, sizeof(double) * nfy(P));
  memcpy(P->bz[s], bz, sizeof(double) * nfz(P));
  int bad;
  P->smax[s] = slice_smax(c, P, s, &bad);
  return bad ? ORC_EUNPHYS : ORC_OK;
}

int orc_set_latest(orc_ctx *c, int ip, int s, double dt_last) {
  if (s < 0 || s >= c->nslot) return ORC_EINVAL;
  c->p[ip].latest = s;
  c->p[ip].dt_last = dt_last;
  return ORC_OK;
}

int orc_get_state(orc_ctx *c, double *U, double *bx, double *by, double *bz) {
  int64_t oU = 0, ox = 0, oy = 0, oz = 0;
  for (int i = 0; i < c->np; i++) {
    opatch *P = &c->p[i];
    int s = P->latest;
    memcpy(U + oU, P->U[s], sizeof(double) * 5 * ncell(P));
    memcpy(bx + ox, P->bx[s], sizeof(double) * nfx(P));
    memcpy(by + oy, P->by[s], sizeof(double) * nfy(P));
    memcpy(bz + oz, P->bz[s], sizeof(double) * nfz(P));
    oU += 5 * ncell(P); ox += nfx(P); oy += nfy(P); oz += nfz(P);
  }
  return ORC_OK;
}

int orc_get_times(orc_ctx *c, double *t, double *dt_last, double *smax) {
  for (int i = 0; i < c->np; i++) {
    opatch *P = &c->p[i];
    if (t) t[i] = P->ts[P->latest];
    if (dt_last) dt_last[i] = P->dt_last;
    if (smax) smax[i] = P->smax[P->latest];
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Guard fill (time interpolation)                                     */
/* ------------------------------------------------------------------ */

/* The stored slices of a patch and the weights that give its values at
 * time t (Sec. 3 A and B): n = 1, a slice at exactly t, copied; n = 2,
 * linear inter- or extrapolation A + w (B - A) between two slices with
 * w = (t - t_a)/(t_b - t_a); n = 3, quadratic (Lagrange) inter- or
 * extrapolation (w_a A + w_b B) + w_c C through three slices.  Slots s[] are
 * ordered from older to newer. */
typedef struct {
  int n;
  int s[3];
  double w[3];
} tpick;

/* Which slices supply time t.  The stored slices, newest first, have
 * strictly decreasing times.  A slice at t is copied.  Past the newest
 * slice (a neighbour that is behind, allowed by the grace of Eq. 1) the
 * newest two (linear) or three (quadratic) are extrapolated.  Otherwise t
 * lies between two consecutive slices, which are interpolated; the
 * quadratic form adds the next older slice, or the next newer one where
 * there is no older one, and stays linear with only two slices. */
static int pick(orc_ctx *c, opatch *Q, double t, tpick *pk) {
  int ns = c->nslot, sl[64], cnt = 0;
  for (int k = 0; k < ns && k < 64; k++) {
    int s = (Q->latest - k + ns) % ns;
    if (isnan(Q->ts[s])) break;
    sl[cnt++] = s;
  }
  for (int k = 0; k < cnt; k++)
    if (Q->ts[sl[k]] == t) {
      pk->n = 1; pk->s[0] = sl[k]; pk->w[0] = 1.0;
      return ORC_OK;
    }
  int ka, kb, kc = -1; /* indices into sl (larger = older) */
  if (t > Q->ts[sl[0]]) {
    if (cnt < 2) return ORC_EBRACKET;
    ka = 1; kb = 0;
    if (c->torder == 2 && cnt >= 3) { kc = 0; kb = 1; ka = 2; }
  } else {
    int k = 1;
    while (k < cnt && !(Q->ts[sl[k]] < t)) k++;
    if (k >= cnt) return ORC_EBRACKET;
    ka = k; kb = k - 1;
    if (c->torder == 2) {
      if (k + 1 < cnt) { kc = k - 1; kb = k; ka = k + 1; }
      else if (k - 2 >= 0) { kc = k - 2; }
    }
  }
  if (kc < 0) {
    double ta = Q->ts[sl[ka]], tb = Q->ts[sl[kb]];
    pk->n = 2; pk->s[0] = sl[ka]; pk->s[1] = sl[kb];
    pk->w[0] = (t - ta) / (tb - ta);
    return ORC_OK;
  }
  double ta = Q->ts[sl[ka]], tb = Q->ts[sl[kb]], tc = Q->ts[sl[kc]];
  pk->n = 3; pk->s[0] = sl[ka]; pk->s[1] = sl[kb]; pk->s[2] = sl[kc];
  pk->w[0] = ((t - tb) * (t - tc)) / ((ta - tb) * (ta - tc));
  pk->w[1] = ((t - ta) * (t - tc)) / ((tb - ta) * (tb - tc));
  pk->w[2] = ((t - ta) * (t - tb)) / ((tc - ta) * (tc - tb));
  return ORC_OK;
}

/* Value at index idx of the array arr[slot] (one array per slice) at the
 * picked time. */
static double tval(double *const *arr, int64_t off, const tpick *pk, int64_t idx) {
  double a = arr[pk->s[0]][off + idx];
  if (pk->n == 1) return a;
  double b = arr[pk->s[1]][off + idx];
  if (pk->n == 2) return a + pk->w[0] * (b - a);
  double cc = arr[pk->s[2]][off + idx];
  return (pk->w[0] * a + pk->w[1] * b) + pk->w[2] * cc;
}

/* Locate the patch of level lev among P's neighbours (or P itself) whose
 * interior holds the level-lev cell g (periodic), and the local cell index
 * there; -1 if none. */
static int owner(orc_ctx *c, opatch *P, int ip, int lev, const int64_t g[3], int loc[3]) {
  for (int q = -1; q < P->nnb; q++) {
    int iq = q < 0 ? ip : P->nb[q];
    opatch *Q = &c->p[iq];
    if (Q->level != lev) continue;
    int in = 1;
    for (int d = 0; d < 3; d++) {
      int64_t r = imod(g[d] - Q->lo[d], c->L[lev][d]);
      if (r >= Q->n[d]) { in = 0; break; }
      loc[d] = (int)r;
    }
    if (in) return iq;
  }
  return -1;
}

/* Conserved values u[5] of level-lev cell g at time t, from the patch of
 * that level that owns it (copied or interpolated in time). */
static int cell_at(orc_ctx *c, opatch *P, int ip, int lev, const int64_t g[3], double t, double u[5]) {
  int loc[3];
  tpick pk;
  int iq = owner(c, P, ip, lev, g, loc);
  if (iq < 0) return ORC_EINVAL;
  opatch *Q = &c->p[iq];
  if (pick(c, Q, t, &pk) != ORC_OK) return ORC_EBRACKET;
  int64_t qc = ncell(Q);
  int64_t id = ((int64_t)loc[2] * Q->n[1] + loc[1]) * Q->n[0] + loc[0];
  for (int q = 0; q < 5; q++) u[q] = tval(Q->U, q * qc, &pk, id);
  return ORC_OK;
}

/* Face along axis ax on the low side of level-lev cell g at time t, from
 * the patch of that level that owns the cell; `up` = 1 takes the face on the
 * cell's high side instead (the same patch owns both). */
static int face_at(orc_ctx *c, opatch *P, int ip, int lev, int ax, const int64_t g[3], int up, double t,
                   double *out) {
  int loc[3];
  tpick pk;
  int iq = owner(c, P, ip, lev, g, loc);
  if (iq < 0) return ORC_EINVAL;
  opatch *Q = &c->p[iq];
  if (pick(c, Q, t, &pk) != ORC_OK) return ORC_EBRACKET;
  loc[ax] += up;
  int qx = Q->n[0], qy = Q->n[1];
  int64_t id = ax == 0 ? ((int64_t)loc[2] * qy + loc[1]) * (qx + 1) + loc[0]
             : ax == 1 ? ((int64_t)loc[2] * (qy + 1) + loc[1]) * qx + loc[0]
                       : ((int64_t)loc[2] * qy + loc[1]) * qx + loc[0];
  double **arr = ax == 0 ? Q->bx : ax == 1 ? Q->by : Q->bz;
  *out = tval(arr, 0, &pk, id);
  return ORC_OK;
}

/* Is level-0 cell C covered by level 1 (its children lie in a level-1
 * patch; level-1 patches cover whole level-0 cells)? */
static int covered(orc_ctx *c, opatch *P, int ip, const int64_t C[3]) {
  int64_t f[3] = {2 * C[0], 2 * C[1], 2 * C[2]};
  int loc[3];
  return owner(c, P, ip, 1, f, loc) >= 0;
}

/* Restriction (Sec. 3 A: guard values in space from a neighbour of other
 * resolution, by conservative averaging): the conserved values of level-0 cell C are the mean of its 8
 * level-1 children, summed z-, y-, x-child in that order. */
static int restrict_cell(orc_ctx *c, opatch *P, int ip, const int64_t C[3], double t, double u[5]) {
  double s[5] = {0, 0, 0, 0, 0}, v[5];
  for (int kz = 0; kz < 2; kz++)
    for (int ky = 0; ky < 2; ky++)
      for (int kx = 0; kx < 2; kx++) {
        int64_t f[3] = {2 * C[0] + kx, 2 * C[1] + ky, 2 * C[2] + kz};
        int rc = cell_at(c, P, ip, 1, f, t, v);
        if (rc) return rc;
        for (int q = 0; q < 5; q++) s[q] = s[q] + v[q];
      }
  for (int q = 0; q < 5; q++) u[q] = 0.125 * s[q];
  return ORC_OK;
}

/* The face along ax on the low side of level-0 cell C: the mean of the 4
 * level-1 faces on it (the children's low faces), the two transverse child
 * offsets looped in z, y, x order. */
static int restrict_face(orc_ctx *c, opatch *P, int ip, int ax, const int64_t C[3], double t, double *out) {
  double s = 0.0, v;
  for (int kz = 0; kz < 2; kz++)
    for (int ky = 0; ky < 2; ky++)
      for (int kx = 0; kx < 2; kx++) {
        int k3[3] = {kx, ky, kz};
        if (k3[ax]) continue;
        int64_t f[3] = {2 * C[0] + kx, 2 * C[1] + ky, 2 * C[2] + kz};
        int rc = face_at(c, P, ip, 1, ax, f, 0, t, &v);
        if (rc) return rc;
        s = s + v;
      }
  *out = 0.25 * s;
  return ORC_OK;
}

/* Prolongation (Sec. 3 A: conservative interpolation from a coarser
 * neighbour): level-1 cell f
 * takes its level-0 parent C's conserved values plus a quarter of the
 * MC-limited slopes of C (one per axis, from C's two level-0 neighbours on
 * that axis), signed by the child's side: u = u_C + (s_x sx + s_y sy +
 * s_z sz)/4.  The 8 children of C average to u_C.  Level-0 values are read
 * as stored, also under the refined region. */
static int prolong_cell(orc_ctx *c, opatch *P, int ip, const int64_t f[3], double t, double u[5]) {
  int64_t C[3] = {fdiv(f[0], 2), fdiv(f[1], 2), fdiv(f[2], 2)};
  double uc[5], ul[5], ur[5], sl[3][5];
  int rc = cell_at(c, P, ip, 0, C, t, uc);
  if (rc) return rc;
  for (int d = 0; d < 3; d++) {
    int64_t Cm[3] = {C[0], C[1], C[2]}, Cp[3] = {C[0], C[1], C[2]};
    Cm[d] -= 1;
    Cp[d] += 1;
    if ((rc = cell_at(c, P, ip, 0, Cm, t, ul))) return rc;
    if ((rc = cell_at(c, P, ip, 0, Cp, t, ur))) return rc;
    for (int q = 0; q < 5; q++) sl[d][q] = mc(uc[q] - ul[q], ur[q] - uc[q]);
  }
  for (int q = 0; q < 5; q++) {
    double a = (f[0] - 2 * C[0]) ? sl[0][q] : -sl[0][q];
    double b = (f[1] - 2 * C[1]) ? sl[1][q] : -sl[1][q];
    double e = (f[2] - 2 * C[2]) ? sl[2][q] : -sl[2][q];
    u[q] = uc[q] + 0.25 * ((a + b) + e);
  }
  return ORC_OK;
}

/* The face along ax on the low side of level-1 cell f, from level 0: a
 * level-1 face on a level-0 face takes that face's value; a level-1 face
 * inside a level-0 cell takes the mean of that cell's two faces along ax.
 * Piecewise constant along the face, so every level-1 cell inside one
 * level-0 cell keeps that cell's divergence. */
static int prolong_face(orc_ctx *c, opatch *P, int ip, int ax, const int64_t f[3], double t, double *out) {
  int64_t C[3] = {fdiv(f[0], 2), fdiv(f[1], 2), fdiv(f[2], 2)};
  double lo, hi;
  int rc = face_at(c, P, ip, 0, ax, C, 0, t, &lo);
  if (rc) return rc;
  if (f[ax] == 2 * C[ax]) { *out = lo; return ORC_OK; }
  if ((rc = face_at(c, P, ip, 0, ax, C, 1, t, &hi))) return rc;
  *out = 0.5 * (lo + hi);
  return ORC_OK;
}

typedef struct {
  int N[3];          /* padded cell counts per axis */
  double *U;         /* [5][Nz][Ny][Nx] */
  double *bx, *by, *bz;
} padded;

#define PC(pd, i, j, k) ((((int64_t)(k) + g) * (pd)->N[1] + ((j) + g)) * (pd)->N[0] + ((i) + g))
#define PFX(pd, i, j, k) ((((int64_t)(k) + g) * (pd)->N[1] + ((j) + g)) * ((pd)->N[0] + 1) + ((i) + g))
#define PFY(pd, i, j, k) ((((int64_t)(k) + g) * ((pd)->N[1] + 1) + ((j) + g)) * (pd)->N[0] + ((i) + g))
#define PFZ(pd, i, j, k) ((((int64_t)(k) + g) * (pd)->N[1] + ((j) + g)) * (pd)->N[0] + ((i) + g))

/* Fill the padded box of patch ip at its current time.  Cell-centred values
 * of guard cells come from the neighbour of the same level owning the cell;
 * on level 0 a guard cell covered by level 1 is restricted from there, and
 * on level 1 a guard cell no level-1 patch owns is prolonged from level 0.
 * A face on one of P's interior cells is P's own; any other face is taken by
 * the same rules from the cell on the face's upper side. */
static int fill_padded(orc_ctx *c, int ip, padded *pd) {
  opatch *P = &c->p[ip];
  int g = c->g, lev = P->level;
  int nx = P->n[0], ny = P->n[1], nz = P->n[2];
  int Nx = nx + 2 * g, Ny = ny + 2 * g, Nz = nz + 2 * g;
  int64_t Nc = (int64_t)Nx * Ny * Nz;
  double t = P->ts[P->latest];
  int s0 = P->latest;
  int64_t nc = ncell(P);
  pd->N[0] = Nx; pd->N[1] = Ny; pd->N[2] = Nz;
  for (int k = -g; k < nz + g; k++)
    for (int j = -g; j < ny + g; j++)
      for (int i = -g; i < nx + g; i++) {
        int64_t pi = PC(pd, i, j, k);
        if (i >= 0 && i < nx && j >= 0 && j < ny && k >= 0 && k < nz) {
          int64_t id = ((int64_t)k * ny + j) * nx + i;
          for (int q = 0; q < 5; q++) pd->U[q * Nc + pi] = P->U[s0][q * nc + id];
          continue;
        }
        int64_t gc[3] = {P->lo[0] + i, P->lo[1] + j, P->lo[2] + k};
        double u[5];
        int loc[3], rc;
        if (lev == 0 && c->nlev > 1 && covered(c, P, ip, gc)) rc = restrict_cell(c, P, ip, gc, t, u);
        else if (owner(c, P, ip, lev, gc, loc) >= 0) rc = cell_at(c, P, ip, lev, gc, t, u);
        else if (lev == 1) rc = prolong_cell(c, P, ip, gc, t, u);
        else rc = ORC_EINVAL;
        if (rc) return rc;
        for (int q = 0; q < 5; q++) pd->U[q * Nc + pi] = u[q];
      }
  /* faces, one axis at a time */
  for (int ax = 0; ax < 3; ax++) {
    int ex = ax == 0, ey = ax == 1, ez = ax == 2;
    for (int k = -g; k < nz + g + ez; k++)
      for (int j = -g; j < ny + g + ey; j++)
        for (int i = -g; i < nx + g + ex; i++) {
          int64_t pi = ax == 0 ? PFX(pd, i, j, k) : ax == 1 ? PFY(pd, i, j, k) : PFZ(pd, i, j, k);
          double *dst = ax == 0 ? pd->bx : ax == 1 ? pd->by : pd->bz;
          int own = (i >= 0 && i < nx + ex && j >= 0 && j < ny + ey && k >= 0 && k < nz + ez);
          if (own) {
            int64_t id = ax == 0 ? ((int64_t)k * ny + j) * (nx + 1) + i
                       : ax == 1 ? ((int64_t)k * (ny + 1) + j) * nx + i
                                 : ((int64_t)k * ny + j) * nx + i;
            dst[pi] = (ax == 0 ? P->bx[s0] : ax == 1 ? P->by[s0] : P->bz[s0])[id];
            continue;
          }
          int64_t gc[3] = {P->lo[0] + i, P->lo[1] + j, P->lo[2] + k};
          int loc[3], rc;
          double v;
          if (lev == 0 && c->nlev > 1 && covered(c, P, ip, gc)) rc = restrict_face(c, P, ip, ax, gc, t, &v);
          else if (owner(c, P, ip, lev, gc, loc) >= 0) rc = face_at(c, P, ip, lev, ax, gc, 0, t, &v);
          else if (lev == 1) rc = prolong_face(c, P, ip, ax, gc, t, &v);
          else rc = ORC_EINVAL;
          if (rc) return rc;
          dst[pi] = v;
        }
  }
  return ORC_OK;
}

/* The padded box of patch ip at its current time, as the update reads it
 * (guard depth g): U[5][Nz][Ny][Nx], bx[Nz][Ny][Nx+1], by[Nz][Ny+1][Nx],
 * bz[Nz+1][Ny][Nx] with N = n + 2g; for checking the guard fill alone. */
int orc_fill_padded(orc_ctx *c, int ip, double *U, double *bx, double *by, double *bz) {
  padded pd;
  pd.U = U; pd.bx = bx; pd.by = by; pd.bz = bz;
  return fill_padded(c, ip, &pd);
}

/* ------------------------------------------------------------------ */
/* One update of one patch                                             */
/* ------------------------------------------------------------------ */

/* Advance patch ip by dt from its current time, writing the new interior
 * state into the given arrays and its signal-speed sum into *smax_out. */
static int update_patch(orc_ctx *c, int ip, double dt, double *oU, double *obx, double *oby, double *obz,
                        double *smax_out, int64_t *nfallback, int64_t *nfloor) {
  opatch *P = &c->p[ip];
  int g = c->g;
  int nx = P->n[0], ny = P->n[1], nz = P->n[2];
  int Nx = nx + 2 * g, Ny = ny + 2 * g, Nz = nz + 2 * g;
  int64_t Nc = (int64_t)Nx * Ny * Nz;
  int64_t Nfx = (int64_t)(Nx + 1) * Ny * Nz, Nfy = (int64_t)Nx * (Ny + 1) * Nz, Nfz = (int64_t)Nx * Ny * (Nz + 1);
  int64_t Ne = (int64_t)(Nx + 1) * (Ny + 1) * (Nz + 1);
  padded pdv, *pd = &pdv;
  pd->U = (double *)malloc(sizeof(double) * 5 * Nc);
  pd->bx = (double *)malloc(sizeof(double) * Nfx);
  pd->by = (double *)malloc(sizeof(double) * Nfy);
  pd->bz = (double *)malloc(sizeof(double) * Nfz);
  double *W = (double *)malloc(sizeof(double) * 8 * Nc);
  double *Ws = (double *)malloc(sizeof(double) * 8 * Nc);
  double *dW = (double *)malloc(sizeof(double) * 24 * Nc);
  double *F[3], *S[3];
  for (int d = 0; d < 3; d++) {
    F[d] = (double *)malloc(sizeof(double) * 5 * Ne);
    S[d] = (double *)malloc(sizeof(double) * 2 * Ne);
  }
  double *E[3], *J[3] = {NULL, NULL, NULL}, *Eni[3] = {NULL, NULL, NULL};
  for (int d = 0; d < 3; d++) E[d] = (double *)malloc(sizeof(double) * Ne);
  int nonideal = c->eta > 0.0 || c->gad > 0.0;
  if (nonideal)
    for (int d = 0; d < 3; d++) {
      J[d] = (double *)malloc(sizeof(double) * Ne);
      Eni[d] = (double *)malloc(sizeof(double) * Ne);
    }
  int rc = fill_padded(c, ip, pd);
  if (rc != ORC_OK) goto done;

  double gamma = c->gamma;
  double dxl = ldexp(c->dx, -P->level);
  double h = 0.5 * dt / dxl;
  double dtdx = dt / dxl;

  /* A4: primitives on every padded cell */
  for (int k = -g; k < nz + g; k++)
    for (int j = -g; j < ny + g; j++)
      for (int i = -g; i < nx + g; i++) {
        int64_t pi = PC(pd, i, j, k);
        double u[5], w8[8];
        for (int q = 0; q < 5; q++) u[q] = pd->U[q * Nc + pi];
        prim(u, pd->bx[PFX(pd, i, j, k)], pd->bx[PFX(pd, i + 1, j, k)], pd->by[PFY(pd, i, j, k)],
             pd->by[PFY(pd, i, j + 1, k)], pd->bz[PFZ(pd, i, j, k)], pd->bz[PFZ(pd, i, j, k + 1)], gamma, w8);
        for (int q = 0; q < 8; q++) W[q * Nc + pi] = w8[q];
      }

  /* A5/A6: limited slopes and the half-step predictor on cells [-1, n] */
  for (int k = -1; k <= nz; k++)
    for (int j = -1; j <= ny; j++)
      for (int i = -1; i <= nx; i++) {
        int64_t pi = PC(pd, i, j, k);
        double w8[8], d3[3][8], ws[8];
        for (int q = 0; q < 8; q++) w8[q] = W[q * Nc + pi];
        for (int d = 0; d < 3; d++) {
          int64_t pm = d == 0 ? PC(pd, i - 1, j, k) : d == 1 ? PC(pd, i, j - 1, k) : PC(pd, i, j, k - 1);
          int64_t pp = d == 0 ? PC(pd, i + 1, j, k) : d == 1 ? PC(pd, i, j + 1, k) : PC(pd, i, j, k + 1);
          for (int q = 0; q < 8; q++) {
            if (q == BX + d) {
              double fl = d == 0 ? pd->bx[PFX(pd, i, j, k)] : d == 1 ? pd->by[PFY(pd, i, j, k)] : pd->bz[PFZ(pd, i, j, k)];
              double fr = d == 0 ? pd->bx[PFX(pd, i + 1, j, k)] : d == 1 ? pd->by[PFY(pd, i, j + 1, k)] : pd->bz[PFZ(pd, i, j, k + 1)];
              d3[d][q] = fr - fl;
            } else {
              double dl = w8[q] - W[q * Nc + pm];
              double dr = W[q * Nc + pp] - w8[q];
              d3[d][q] = mc(dl, dr);
            }
          }
        }
        predict(w8, d3[0], d3[1], d3[2], gamma, h, ws);
        /* positivity fallback: any face state with rho <= 0 or p <= 0 */
        int bad = 0;
        for (int d = 0; d < 3; d++) {
          double rp = ws[RHO] + 0.5 * d3[d][RHO], rm = ws[RHO] - 0.5 * d3[d][RHO];
          double pp_ = ws[PR] + 0.5 * d3[d][PR], pm_ = ws[PR] - 0.5 * d3[d][PR];
          if (!(rp > 0.0) || !(rm > 0.0) || !(pp_ > 0.0) || !(pm_ > 0.0)) bad = 1;
        }
        if (bad) {
          (*nfallback)++;
          for (int d = 0; d < 3; d++)
            for (int q = 0; q < 8; q++) d3[d][q] = 0.0;
          for (int q = 0; q < 8; q++) ws[q] = w8[q];
        }
        for (int q = 0; q < 8; q++) Ws[q * Nc + pi] = ws[q];
        for (int d = 0; d < 3; d++)
          for (int q = 0; q < 8; q++) dW[(d * 8 + q) * Nc + pi] = d3[d][q];
      }

#define EI(i, j, k) ((((int64_t)(k) + g) * (Ny + 1) + ((j) + g)) * (Nx + 1) + ((i) + g))
  /* A7: HLL (or HLLD) fluxes.  Face index i on axis d is the face at i-1/2 between
   * cells i-1 and i; computed for all faces whose two cells lie in [-1, n]. */
  for (int d = 0; d < 3; d++) {
    int ex = d == 0, ey = d == 1, ez = d == 2;
    for (int k = ez ? 0 : -1; k <= nz; k++)
      for (int j = ey ? 0 : -1; j <= ny; j++)
        for (int i = ex ? 0 : -1; i <= nx; i++) {
          int64_t pr = PC(pd, i, j, k);
          int64_t pl = PC(pd, i - ex, j - ey, k - ez);
          double WL[8], WR[8], f7[7], s2[2];
          for (int q = 0; q < 8; q++) {
            WL[q] = Ws[q * Nc + pl] + 0.5 * dW[(d * 8 + q) * Nc + pl];
            WR[q] = Ws[q * Nc + pr] - 0.5 * dW[(d * 8 + q) * Nc + pr];
          }
          if (c->riemann) hlld(WL, WR, d, gamma, f7, s2);
          else hll(WL, WR, d, gamma, f7, s2);
          int64_t e = EI(i, j, k);
          for (int q = 0; q < 5; q++) F[d][q * Ne + e] = f7[q];
          S[d][e] = s2[0];
          S[d][Ne + e] = s2[1];
        }
  }

  /* A8: edge EMFs.  E[e] at index (i,j,k) is the edge along axis e located at
   * the low corner of cell (i,j,k) in the two other axes. */
  for (int e = 0; e < 3; e++) {
    int a = (e + 1) % 3, b = (e + 2) % 3;
    int lo3[3] = {0, 0, 0}, hi3[3] = {nx, ny, nz};
    hi3[a] += 1; hi3[b] += 1;
    for (int k = lo3[2]; k < hi3[2]; k++)
      for (int j = lo3[1]; j < hi3[1]; j++)
        for (int i = lo3[0]; i < hi3[0]; i++) {
          int o[3] = {i, j, k};
          int cll[3], crl[3], clr[3], crr[3];
          for (int q = 0; q < 3; q++) { cll[q] = crl[q] = clr[q] = crr[q] = o[q]; }
          cll[a] -= 1; cll[b] -= 1;
          crl[b] -= 1;
          clr[a] -= 1;
          int *cs[4] = {cll, crl, clr, crr};
          double sa_[4] = {+0.5, -0.5, +0.5, -0.5};
          double sb_[4] = {+0.5, +0.5, -0.5, -0.5};
          double Wc[4][8];
          for (int r = 0; r < 4; r++) {
            int64_t pi = PC(pd, cs[r][0], cs[r][1], cs[r][2]);
            for (int q = 0; q < 8; q++) {
              double ws = Ws[q * Nc + pi];
              double da = dW[(a * 8 + q) * Nc + pi];
              double db = dW[(b * 8 + q) * Nc + pi];
              double v = sa_[r] > 0 ? ws + 0.5 * da : ws - 0.5 * da;
              Wc[r][q] = sb_[r] > 0 ? v + 0.5 * db : v - 0.5 * db;
            }
          }
          /* a-faces touching the edge: face index o on axis a, cells b-1 and b */
          int fa1[3] = {i, j, k}, fb1[3] = {i, j, k};
          fa1[b] -= 1;
          fb1[a] -= 1;
          int64_t ea0 = EI(fa1[0], fa1[1], fa1[2]), ea1 = EI(i, j, k);
          int64_t eb0 = EI(fb1[0], fb1[1], fb1[2]), eb1 = EI(i, j, k);
          double apa = fmax(0.0, fmax(S[a][Ne + ea0], S[a][Ne + ea1]));
          double ama = fmax(0.0, fmax(-S[a][ea0], -S[a][ea1]));
          double apb = fmax(0.0, fmax(S[b][Ne + eb0], S[b][Ne + eb1]));
          double amb = fmax(0.0, fmax(-S[b][eb0], -S[b][eb1]));
          E[e][EI(i, j, k)] = emf(Wc[0], Wc[1], Wc[2], Wc[3], e, apa, ama, apb, amb);
        }
  }

  /* Non-ideal EMFs (Sec. 4.3), from the state at the start of the step.
   * Currents live on the edges, as the EMFs do: J_e at edge o (axis e, low
   * corner of cell o in a = e+1 and b = e+2) is the discrete curl of the
   * four faces around it, (f_b(o) - f_b(o - a)) - (f_a(o) - f_a(o - b)), over
   * dx.  E_Ohm = eta J_e (Eq. 8).  E_AD = (J B^2 - B (B.J)) / (gamma_AD rho
   * rho_i), which is -v_D x B of Eqs. 5-6, with the edge's B_a and B_b the
   * means of the two faces on the edge, B_e and rho the means over the four
   * cells around it (cell-centred B), and J_a, J_b the means of the four
   * nearest a- and b-edges.  The EMF of the induction equation becomes
   * E_ideal + E_Ohm + E_AD, and the energy flux through each face gains the
   * Poynting flux (E_Ohm + E_AD) x B (edge EMFs and cell-centred B averaged
   * to the face), so total energy stays conserved and the magnetic energy
   * the terms remove, the heating Q of Eqs. 9 and 13, goes into the
   * internal energy. */
  if (nonideal) {
    double idx = 1.0 / dxl;
#define FACE(ax, i, j, k) ((ax) == 0 ? pd->bx[PFX(pd, i, j, k)] : (ax) == 1 ? pd->by[PFY(pd, i, j, k)] : pd->bz[PFZ(pd, i, j, k)])
    for (int e = 0; e < 3; e++) {
      int a = (e + 1) % 3, b = (e + 2) % 3;
      for (int k = -1; k <= nz + 1; k++)
        for (int j = -1; j <= ny + 1; j++)
          for (int i = -1; i <= nx + 1; i++) {
            int o[3] = {i, j, k}, oa[3] = {i, j, k}, ob[3] = {i, j, k};
            oa[a] -= 1;
            ob[b] -= 1;
            double dbb = FACE(b, o[0], o[1], o[2]) - FACE(b, oa[0], oa[1], oa[2]);
            double dba = FACE(a, o[0], o[1], o[2]) - FACE(a, ob[0], ob[1], ob[2]);
            J[e][EI(i, j, k)] = (dbb - dba) * idx;
          }
    }
    for (int e = 0; e < 3; e++) {
      int a = (e + 1) % 3, b = (e + 2) % 3;
      int hi3[3] = {nx, ny, nz};
      hi3[a] += 1; hi3[b] += 1;
      for (int k = 0; k < hi3[2]; k++)
        for (int j = 0; j < hi3[1]; j++)
          for (int i = 0; i < hi3[0]; i++) {
            int o[3] = {i, j, k};
            double en = 0.0;
            if (c->eta > 0.0) en = c->eta * J[e][EI(i, j, k)];
            if (c->gad > 0.0) {
              int oa[3] = {i, j, k}, ob[3] = {i, j, k}, oab[3] = {i, j, k};
              oa[a] -= 1; ob[b] -= 1; oab[a] -= 1; oab[b] -= 1;
              int64_t c0 = PC(pd, o[0], o[1], o[2]), ca = PC(pd, oa[0], oa[1], oa[2]);
              int64_t cb = PC(pd, ob[0], ob[1], ob[2]), cab = PC(pd, oab[0], oab[1], oab[2]);
              double Ba = 0.5 * (FACE(a, o[0], o[1], o[2]) + FACE(a, ob[0], ob[1], ob[2]));
              double Bb = 0.5 * (FACE(b, o[0], o[1], o[2]) + FACE(b, oa[0], oa[1], oa[2]));
              double Be = 0.25 * ((W[(BX + e) * Nc + c0] + W[(BX + e) * Nc + ca]) +
                                  (W[(BX + e) * Nc + cb] + W[(BX + e) * Nc + cab]));
              double re = 0.25 * ((W[RHO * Nc + c0] + W[RHO * Nc + ca]) + (W[RHO * Nc + cb] + W[RHO * Nc + cab]));
              /* a-edges at a = o_a - 1, o_a and e = o_e, o_e + 1; b-edges alike */
              int ae[3] = {i, j, k}, aae[3] = {i, j, k}, be[3] = {i, j, k}, bbe[3] = {i, j, k};
              ae[e] += 1; aae[a] -= 1; aae[e] += 1;
              be[e] += 1; bbe[b] -= 1; bbe[e] += 1;
              double Ja = 0.25 * ((J[a][EI(i, j, k)] + J[a][EI(oa[0], oa[1], oa[2])]) +
                                  (J[a][EI(ae[0], ae[1], ae[2])] + J[a][EI(aae[0], aae[1], aae[2])]));
              double Jb = 0.25 * ((J[b][EI(i, j, k)] + J[b][EI(ob[0], ob[1], ob[2])]) +
                                  (J[b][EI(be[0], be[1], be[2])] + J[b][EI(bbe[0], bbe[1], bbe[2])]));
              double Je = J[e][EI(i, j, k)];
              double B2 = (Be * Be + Ba * Ba) + Bb * Bb;
              double BJ = (Be * Je + Ba * Ja) + Bb * Jb;
              en = en + (Je * B2 - Be * BJ) / ((c->gad * re) * c->rhoi);
            }
            Eni[e][EI(i, j, k)] = en;
            E[e][EI(i, j, k)] = E[e][EI(i, j, k)] + en;
          }
    }
    /* Poynting flux of the non-ideal EMF through the update's faces */
    for (int d = 0; d < 3; d++) {
      int a = (d + 1) % 3, b = (d + 2) % 3;
      int hi3[3] = {nx, ny, nz};
      hi3[d] += 1;
      for (int k = 0; k < hi3[2]; k++)
        for (int j = 0; j < hi3[1]; j++)
          for (int i = 0; i < hi3[0]; i++) {
            int ob[3] = {i, j, k}, oa[3] = {i, j, k}, od[3] = {i, j, k};
            ob[b] += 1; oa[a] += 1; od[d] -= 1;
            double Ea = 0.5 * (Eni[a][EI(i, j, k)] + Eni[a][EI(ob[0], ob[1], ob[2])]);
            double Eb = 0.5 * (Eni[b][EI(i, j, k)] + Eni[b][EI(oa[0], oa[1], oa[2])]);
            int64_t cl = PC(pd, od[0], od[1], od[2]), cr = PC(pd, i, j, k);
            double Ba = 0.5 * (W[(BX + a) * Nc + cl] + W[(BX + a) * Nc + cr]);
            double Bb = 0.5 * (W[(BX + b) * Nc + cl] + W[(BX + b) * Nc + cr]);
            int64_t f = 4 * Ne + EI(i, j, k);
            F[d][f] = F[d][f] + (Ea * Bb - Eb * Ba);
          }
    }
#undef FACE
  }

  /* A9: conservative update of U and constrained-transport update of b */
  int64_t nc = ncell(P);
  const double *U0 = P->U[P->latest];
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        int64_t id = ((int64_t)k * ny + j) * nx + i;
        for (int q = 0; q < 5; q++) {
          double fxp = F[0][q * Ne + EI(i + 1, j, k)], fxm = F[0][q * Ne + EI(i, j, k)];
          double fyp = F[1][q * Ne + EI(i, j + 1, k)], fym = F[1][q * Ne + EI(i, j, k)];
          double fzp = F[2][q * Ne + EI(i, j, k + 1)], fzm = F[2][q * Ne + EI(i, j, k)];
          oU[q * nc + id] = U0[q * nc + id] - dtdx * ((fxp - fxm) + (fyp - fym) + (fzp - fzm));
        }
      }
  const double *bx0 = P->bx[P->latest], *by0 = P->by[P->latest], *bz0 = P->bz[P->latest];
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i <= nx; i++) {
        int64_t id = ((int64_t)k * ny + j) * (nx + 1) + i;
        obx[id] = bx0[id] - dtdx * ((E[2][EI(i, j + 1, k)] - E[2][EI(i, j, k)]) - (E[1][EI(i, j, k + 1)] - E[1][EI(i, j, k)]));
      }
  for (int k = 0; k < nz; k++)
    for (int j = 0; j <= ny; j++)
      for (int i = 0; i < nx; i++) {
        int64_t id = ((int64_t)k * (ny + 1) + j) * nx + i;
        oby[id] = by0[id] - dtdx * ((E[0][EI(i, j, k + 1)] - E[0][EI(i, j, k)]) - (E[2][EI(i + 1, j, k)] - E[2][EI(i, j, k)]));
      }
  for (int k = 0; k <= nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        int64_t id = ((int64_t)k * ny + j) * nx + i;
        obz[id] = bz0[id] - dtdx * ((E[1][EI(i + 1, j, k)] - E[1][EI(i, j, k)]) - (E[0][EI(i, j + 1, k)] - E[0][EI(i, j, k)]));
      }
#undef EI

  /* A10: signal speed of the new state, and the positivity check */
  {
    double m = 0.0;
    int bad = 0;
    for (int k = 0; k < nz; k++)
      for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
          int64_t id = ((int64_t)k * ny + j) * nx + i;
          double u[5], w8[8];
          for (int q = 0; q < 5; q++) u[q] = oU[q * nc + id];
          *nfloor += prim(u, obx[((int64_t)k * ny + j) * (nx + 1) + i], obx[((int64_t)k * ny + j) * (nx + 1) + i + 1],
                          oby[((int64_t)k * (ny + 1) + j) * nx + i], oby[((int64_t)k * (ny + 1) + j + 1) * nx + i],
                          obz[((int64_t)k * ny + j) * nx + i], obz[((int64_t)(k + 1) * ny + j) * nx + i], gamma, w8);
          if (!(w8[RHO] > 0.0) || !(w8[PR] > 0.0)) bad = 1;
          double ir = 1.0 / w8[RHO];
          double cx = cfast(gamma, ir, w8[PR], w8[BX], w8[BY], w8[BZ]);
          double cy = cfast(gamma, ir, w8[PR], w8[BY], w8[BZ], w8[BX]);
          double cz = cfast(gamma, ir, w8[PR], w8[BZ], w8[BX], w8[BY]);
          double sum = (fabs(w8[VX]) + cx) + (fabs(w8[VY]) + cy) + (fabs(w8[VZ]) + cz);
          sum = fmax(sum, nonideal_speed(c, w8, dxl));
          if (sum > m) m = sum;
        }
    *smax_out = m;
    if (bad) rc = ORC_EUNPHYS;
  }

done:
  free(pd->U); free(pd->bx); free(pd->by); free(pd->bz);
  free(W); free(Ws); free(dW);
  for (int d = 0; d < 3; d++) { free(F[d]); free(S[d]); free(E[d]); free(J[d]); free(Eni[d]); }
  return rc;
}

/* ------------------------------------------------------------------ */
/* Time steps, readiness and the dispatcher                            */
/* ------------------------------------------------------------------ */

/* May patch ip overwrite its oldest slice?  Not while a neighbour that may
 * be updated before ip's next slice exists (its time at most ip's time plus
 * g times ip's last step) still takes values from that slice.  With g = 0
 * this never binds: a ready patch is at or behind every neighbour, and
 * neighbours at or past its newest slice read only its newest two (three,
 * quadratic) slices.  An empty slot is always free. */
static int slot_free(orc_ctx *c, int ip) {
  opatch *P = &c->p[ip];
  int oldest = (P->latest + 1) % c->nslot;
  if (isnan(P->ts[oldest])) return 1;
  double lim = P->ts[P->latest] + c->grace * P->dt_last;
  for (int q = 0; q < P->nnb; q++) {
    opatch *Q = &c->p[P->nb[q]];
    double tq = Q->ts[Q->latest];
    if (!(tq <= lim)) continue;
    tpick pk;
    if (pick(c, P, tq, &pk) != ORC_OK) continue;
    for (int k = 0; k < pk.n; k++)
      if (pk.s[k] == oldest) return 0;
  }
  return 1;
}

/* Eq. (1): ready iff t_self < t_end and t_self <= t_nbor + g dt_nbor for all
 * neighbours (dt_nbor: the neighbour's last step, 0 before its first), and,
 * with g > 0, the patch's oldest slice is free (slot_free). */
static int ready(orc_ctx *c, int ip, double t_end) {
  opatch *P = &c->p[ip];
  double t = P->ts[P->latest];
  if (P->virt || !(t < t_end)) return 0;
  for (int q = 0; q < P->nnb; q++) {
    opatch *Q = &c->p[P->nb[q]];
    if (!(t <= Q->ts[Q->latest] + c->grace * Q->dt_last)) return 0;
  }
  if (c->grace > 0.0 && !slot_free(c, ip)) return 0;
  return 1;
}

/* Local Courant step of patch ip at its time, quantised to a power of two,
 * capped by dt_max, halved until it divides the time, clipped to t_end.
 * The signal speed is the largest over the patch's newest slice and every
 * neighbour slice that its guard fill reads. */
static int patch_dt(orc_ctx *c, int ip, double t_end, double *dt_out) {
  opatch *P = &c->p[ip];
  double t = P->ts[P->latest];
  double M = P->smax[P->latest];
  for (int q = 0; q < P->nnb; q++) {
    opatch *Q = &c->p[P->nb[q]];
    tpick pk;
    if (pick(c, Q, t, &pk) != ORC_OK) return ORC_EBRACKET;
    for (int k = 0; k < pk.n; k++) M = fmax(M, Q->smax[pk.s[k]]);
  }
  double dtc = c->cfl * ldexp(c->dx, -P->level) / M;
  double dt = pow2_floor(dtc);
  if (c->dt_max > 0.0 && dt > c->dt_max) dt = c->dt_max;
  while (fmod(t, dt) != 0.0) dt = dt * 0.5;
  if (dt > t_end - t) dt = t_end - t;
  *dt_out = dt;
  return ORC_OK;
}

int orc_patch_dt(orc_ctx *c, int ip, double t_end, double *dt) { return patch_dt(c, ip, t_end, dt); }

static void sched_push(orc_ctx *c, int ip, double t, double dt) {
  if (c->nsched == c->capsched) {
    c->capsched = c->capsched ? 2 * c->capsched : 1024;
    c->s_patch = (int64_t *)realloc(c->s_patch, sizeof(int64_t) * c->capsched);
    c->s_t = (double *)realloc(c->s_t, sizeof(double) * c->capsched);
    c->s_dt = (double *)realloc(c->s_dt, sizeof(double) * c->capsched);
  }
  c->s_patch[c->nsched] = ip;
  c->s_t[c->nsched] = t;
  c->s_dt[c->nsched] = dt;
  c->nsched++;
}

static void publish(orc_ctx *c, int ip, double dt, double smax) {
  opatch *P = &c->p[ip];
  double t = P->ts[P->latest];
  int ns = (P->latest + 1) % c->nslot;
  P->ts[ns] = t + dt;
  P->smax[ns] = smax;
  P->latest = ns;
  P->dt_last = dt;
  sched_push(c, ip, t, dt);
  c->n_updates++;
  c->n_cells += ncell(P);
}

/* Compute one update of patch ip by dt into caller arrays, without
 * publishing it (reproduces a single update for sampled comparisons). */
int orc_update_patch(orc_ctx *c, int ip, double dt, double *U, double *bx, double *by, double *bz, double *smax) {
  int64_t nf = 0, nfl = 0;
  return update_patch(c, ip, dt, U, bx, by, bz, smax, &nf, &nfl);
}

/* One sweep: snapshot every time, collect the ready set R, update every
 * patch of R from the pre-sweep slices, then publish them all. */
static int sweep(orc_ctx *c, double t_end, int *nready) {
  int np = c->np;
  int *R = (int *)malloc(sizeof(int) * np);
  double *dt = (double *)malloc(sizeof(double) * np);
  double *sm = (double *)malloc(sizeof(double) * np);
  int nr = 0, rc = ORC_OK;
  for (int i = 0; i < np; i++)
    if (ready(c, i, t_end)) R[nr++] = i;
  *nready = nr;
  if (nr == 0) goto out;
  for (int r = 0; r < nr; r++) {
    rc = patch_dt(c, R[r], t_end, &dt[r]);
    if (rc) goto out;
  }
  if (c->time_mode == 0) {
    double m = dt[0];
    for (int r = 1; r < nr; r++) m = fmin(m, dt[r]);
    for (int r = 0; r < nr; r++) dt[r] = m;
  }
  int64_t nfb = 0, nfl = 0;
  int err = ORC_OK;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : nfb, nfl)
  for (int r = 0; r < nr; r++) {
    opatch *P = &c->p[R[r]];
    int ns = (P->latest + 1) % c->nslot;
    int64_t f = 0, fl = 0;
    int e = update_patch(c, R[r], dt[r], P->U[ns], P->bx[ns], P->by[ns], P->bz[ns], &sm[r], &f, &fl);
    nfb += f;
    nfl += fl;
    if (e) {
#pragma omp critical
      err = e;
    }
  }
  c->n_fallback += nfb;
  c->n_floor += nfl;
  if (err) { rc = err; goto out; }
  for (int r = 0; r < nr; r++) publish(c, R[r], dt[r], sm[r]);
  c->n_sweeps++;
out:
  free(R); free(dt); free(sm);
  return rc;
}

/* Time-sorted ready queue (the paper's first dispatcher mode, run on one
 * thread): pop the oldest ready patch (ties by index), update and publish
 * it, then re-check it and its neighbours and queue any that became ready. */
static int queue_run(orc_ctx *c, double t_end) {
  int np = c->np;
  char *queued = (char *)calloc(np, 1);
  int rc = ORC_OK;
  for (int i = 0; i < np; i++) queued[i] = (char)ready(c, i, t_end);
  for (;;) {
    int best = -1;
    for (int i = 0; i < np; i++) {
      if (!queued[i]) continue;
      if (best < 0) { best = i; continue; }
      double ti = c->p[i].ts[c->p[i].latest], tb = c->p[best].ts[c->p[best].latest];
      if (ti < tb) best = i;
    }
    if (best < 0) break;
    queued[best] = 0;
    opatch *P = &c->p[best];
    double dt, sm;
    rc = patch_dt(c, best, t_end, &dt);
    if (rc) break;
    int ns = (P->latest + 1) % c->nslot;
    int64_t f = 0, fl = 0;
    rc = update_patch(c, best, dt, P->U[ns], P->bx[ns], P->by[ns], P->bz[ns], &sm, &f, &fl);
    c->n_fallback += f;
    c->n_floor += fl;
    if (rc) break;
    publish(c, best, dt, sm);
    if (!queued[best] && ready(c, best, t_end)) queued[best] = 1;
    for (int q = 0; q < P->nnb; q++) {
      int iq = P->nb[q];
      if (!queued[iq] && ready(c, iq, t_end)) queued[iq] = 1;
    }
  }
  free(queued);
  if (rc == ORC_OK) {
    for (int i = 0; i < np; i++)
      if (c->p[i].ts[c->p[i].latest] < t_end) { rc = ORC_EDEADLOCK; break; }
  }
  return rc;
}

/* Advance until every patch has reached t_end, or until max_sweeps sweeps
 * have run (sweep dispatcher; <= 0 means no limit).  In global time-step
 * mode every sweep is one step of the whole domain with the smallest patch
 * step. */
int orc_advance(orc_ctx *c, double t_end, int64_t max_sweeps) {
  int rc = ORC_OK;
  if (!(t_end < INFINITY) && (max_sweeps <= 0 || (c->time_mode == 1 && c->disp_mode == 0))) {
    snprintf(c->err, sizeof c->err, "an unbounded advance needs a finite t_end or a sweep limit");
    return ORC_EINVAL;
  }
  if (c->time_mode == 1 && c->disp_mode == 0) {
    if (c->nvirt) {
      snprintf(c->err, sizeof c->err, "a context with virtual patches advances by sweeps");
      return ORC_EINVAL;
    }
    rc = queue_run(c, t_end);
  } else {
    for (int64_t s = 0; max_sweeps <= 0 || s < max_sweeps; s++) {
      int nr;
      rc = sweep(c, t_end, &nr);
      if (rc) break;
      if (nr == 0) {
        if (c->nvirt == 0)
          for (int i = 0; i < c->np; i++)
            if (c->p[i].ts[c->p[i].latest] < t_end) { rc = ORC_EDEADLOCK; break; }
        break;
      }
    }
  }
  if (rc) {
    c->status = rc;
    if (!c->err[0]) snprintf(c->err, sizeof c->err, "advance failed with code %d", rc);
  }
  return rc;
}

int64_t orc_get_schedule(orc_ctx *c, int64_t *patch, double *t, double *dt, int64_t cap) {
  int64_t n = c->nsched < cap ? c->nsched : cap;
  if (patch) memcpy(patch, c->s_patch, sizeof(int64_t) * n);
  if (t) memcpy(t, c->s_t, sizeof(double) * n);
  if (dt) memcpy(dt, c->s_dt, sizeof(double) * n);
  return c->nsched;
}

void orc_stats(orc_ctx *c, int64_t *out) {
  out[0] = c->n_updates;
  out[1] = c->n_cells;
  out[2] = c->n_sweeps;
  out[3] = c->n_fallback;
  out[4] = c->n_floor;
}

/* ------------------------------------------------------------------ */
/* Diagnostics: compensated sums and div B                              */
/* ------------------------------------------------------------------ */
typedef struct { double s, c; } nsum;
static void nadd(nsum *a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}

/* Every patch's cells count with their own level's cell volume (with two
 * levels, level-0 cells under the refined region count too).
 * out[0..4]: volume integrals of rho, m_x, m_y, m_z, E (Neumaier sums);
 * out[5..7]: volume integrals of the face fields, each face counted once
 * (the low face of every cell); out[8]: max over cells of |sum_d Delta_d b|;
 * out[9]: max |b| over faces. */
void orc_diagnostics(orc_ctx *c, double *out) {
  nsum acc[8];
  memset(acc, 0, sizeof acc);
  double mdiv = 0.0, mb = 0.0;
  for (int ip = 0; ip < c->np; ip++) {
    opatch *P = &c->p[ip];
    if (P->virt) continue; /* another process owns it and counts it */
    double dxl = ldexp(c->dx, -P->level);
    double dV = dxl * dxl * dxl;
    int s = P->latest, nx = P->n[0], ny = P->n[1], nz = P->n[2];
    int64_t nc = ncell(P);
    for (int k = 0; k < nz; k++)
      for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
          int64_t id = ((int64_t)k * ny + j) * nx + i;
          for (int q = 0; q < 5; q++) nadd(&acc[q], P->U[s][q * nc + id] * dV);
          double bxl = P->bx[s][((int64_t)k * ny + j) * (nx + 1) + i];
          double bxr = P->bx[s][((int64_t)k * ny + j) * (nx + 1) + i + 1];
          double byl = P->by[s][((int64_t)k * (ny + 1) + j) * nx + i];
          double byr = P->by[s][((int64_t)k * (ny + 1) + j + 1) * nx + i];
          double bzl = P->bz[s][((int64_t)k * ny + j) * nx + i];
          double bzr = P->bz[s][((int64_t)(k + 1) * ny + j) * nx + i];
          nadd(&acc[5], bxl * dV);
          nadd(&acc[6], byl * dV);
          nadd(&acc[7], bzl * dV);
          double dv = (bxr - bxl) + (byr - byl) + (bzr - bzl);
          if (fabs(dv) > mdiv) mdiv = fabs(dv);
          if (fabs(bxl) > mb) mb = fabs(bxl);
          if (fabs(byl) > mb) mb = fabs(byl);
          if (fabs(bzl) > mb) mb = fabs(bzl);
        }
  }
  for (int q = 0; q < 8; q++) out[q] = acc[q].s + acc[q].c;
  out[8] = mdiv;
  out[9] = mb;
}

/* ------------------------------------------------------------------ */
/* Several processes (Sec. 3 C, the MPI process view)                   */
/* ------------------------------------------------------------------ */
/* A process holds the patches it owns and 'virtual' copies of the patches
 * other processes own next to them.  owned[i] = 1 for an owned patch, 0 for
 * a virtual one.  A virtual patch is never updated here; each new state of
 * it arrives as a package (its interior and its time parameters) that the
 * owner sends after updating it, and is stored like a new time slice.
 * Every sweep runs here only over the owned patches.  Local time steps with
 * g = 0 only: a global step is a minimum over all processes, and with g > 0
 * a slice's lifetime depends on neighbours held elsewhere. */
int orc_set_owned(orc_ctx *c, const int8_t *owned) {
  int nv = 0;
  for (int i = 0; i < c->np; i++) {
    c->p[i].virt = owned[i] ? 0 : 1;
    nv += c->p[i].virt;
  }
  if (nv && (c->time_mode != 1 || c->grace > 0.0 || c->nlev > 1)) {
    for (int i = 0; i < c->np; i++) c->p[i].virt = 0;
    snprintf(c->err, sizeof c->err, "virtual patches need local steps, g = 0 and one level");
    return ORC_EINVAL;
  }
  c->nvirt = nv;
  return ORC_OK;
}

/* The package of patch ip: its newest slice (U, bx, by, bz in the
 * dsp_set_state layout of one patch) and meta = (time of that slice, the
 * patch's last step, the slice's signal speed). */
int orc_get_newest(orc_ctx *c, int ip, double *U, double *bx, double *by, double *bz, double *meta) {
  if (ip < 0 || ip >= c->np) return ORC_EINVAL;
  opatch *P = &c->p[ip];
  int s = P->latest;
  memcpy(U, P->U[s], sizeof(double) * 5 * ncell(P));
  memcpy(bx, P->bx[s], sizeof(double) * nfx(P));
  memcpy(by, P->by[s], sizeof(double) * nfy(P));
  memcpy(bz, P->bz[s], sizeof(double) * nfz(P));
  meta[0] = P->ts[s];
  meta[1] = P->dt_last;
  meta[2] = P->smax[s];
  return ORC_OK;
}

/* Store a received package as the newest slice of virtual patch ip (in the
 * slot after its newest, as an update would). */
int orc_push_slice(orc_ctx *c, int ip, const double *U, const double *bx, const double *by, const double *bz,
                   const double *meta) {
  if (ip < 0 || ip >= c->np || !c->p[ip].virt) return ORC_EINVAL;
  opatch *P = &c->p[ip];
  int s = (P->latest + 1) % c->nslot;
  memcpy(P->U[s], U, sizeof(double) * 5 * ncell(P));
  memcpy(P->bx[s], bx, sizeof(double) * nfx(P));
  memcpy(P->by[s], by, sizeof(double) * nfy(P));
  memcpy(P->bz[s], bz, sizeof(double) * nfz(P));
  P->ts[s] = meta[0];
  P->dt_last = meta[1];
  P->smax[s] = meta[2];
  P->latest = s;
  return ORC_OK;
}
