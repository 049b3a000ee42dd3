/*
 * tmm_oracle.c -- plain, slow, FP64 CPU statement of the Transport Matrix Method
 * year map of Metos3D (Piwonski & Slawig, "The Idea and Concept of Metos3D",
 * arXiv:1410.0204).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library is checked
 * against.  The library never links, loads or calls it, and it shares no code, header,
 * table or constant with the library; only the tests, the smoke check and the CPU
 * baseline leg of the benchmark use it.
 *
 * What it computes, in the paper's order and notation:
 *   Section 3:     y_{i+1} = A_imp,i ( A_exp,i y_i + q_i(y_i, u) ),  i = 0 .. n_step-1,
 *                  with twelve monthly explicit and twelve monthly implicit matrices,
 *                  linearly interpolated in time;
 *   Section 4:     the year map phi, y(T) = phi(y(0)), n_step = 2880 steps per year;
 *   Section 2.2.1: the PO4-DOP source-minus-sink term q (two tracers, here "N-DOP");
 *   Section 2.2.2: the PO4-DOP-PHY model (three tracers), and two models the batched
 *                  ensemble mixes in: N (PO4 alone) and NPZD-DOP (five tracers), stated
 *                  where they are defined below;
 *   Section 5:     the per-water-column model interface bgc(...), column-local, 360-day
 *                  year, tracer array y(nlayer, ntracer) with the layer index fastest.
 *
 * Readings taken where the paper is silent (each restated where it is used):
 *   R1  the model returns the increment over one ocean step, dt * q for one internal
 *       step, so that y_{i+1} = A_imp (A_exp y_i + dt q(y_i));
 *   R2  with nsub internal model steps (the paper's runs use eight) the increment is
 *       y^(nsub) - y^(0) of nsub explicit Euler steps of length dt/nsub, all using the
 *       forcing passed for the start of the ocean step;
 *   R3  monthly matrix m sits at mid-month, t = (m + 1/2)/12, wrapping from December to
 *       January; both matrices and forcing are taken at the start of the step,
 *       t_j = j / n_step;
 *   R4  the stored monthly implicit matrices themselves are interpolated;
 *   R5  remineralisation of the sinking flux is a source, (F(z_top) - F(z_bot)) / h;
 *   R6  the export integral is the sum over the euphotic layers of f_k h_k; light is
 *       evaluated at the layer centre depth d_k, the flux at layer interfaces;
 *   R7  the flux reaching a column's bottom interface is deposited in its bottom layer
 *       (F(z_bot) = 0 there); a column with no aphotic layer keeps its export in its
 *       bottom layer;
 *   R8  I_SWR is the daily-mean top-of-atmosphere insolation of a circular orbit,
 *       sigma_PAR = 0.4, sigma_ice = 0;
 *   R9  alpha is given per day (times 360 per year), lambda per year, time in years.
 *   R10 the N model is the PO4-DOP model without DOP: all production is exported;
 *   R11 PO4-DOP-PHY rates are per day; the phytoplankton losses of the euphotic zone and
 *       of the whole column feed DOP, and the grazed fraction f_3 = sigma_3 f_1 splits
 *       into DOP (sigma_2) and export (1 - sigma_2), as the PO4-DOP production does;
 *   R12 NPZD-DOP, which the paper does not define, extends PO4-DOP-PHY conservatively:
 *       zooplankton graze phytoplankton with a Holling type II response, and detritus
 *       sinks with a fixed speed (first-order upwind fluxes, none through the sea floor).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MODEL_NONE 0
#define ORACLE_MODEL_N 1
#define ORACLE_MODEL_NDOP 2
#define ORACLE_MODEL_PHY 3
#define ORACLE_MODEL_NPZD 5
#define ORACLE_MAX_LAYER 256
#define ORACLE_MAX_TRACER 8

typedef struct {
    int n;                      /* wet cells */
    int ncol;                   /* water columns */
    int nnz;                    /* nonzeros of one explicit matrix */
    int nmonth;                 /* monthly matrices (12) */
    int nstep;                  /* steps per model year (2880) */
    const int *col_start;       /* [ncol+1] first cell of each column, surface first */
    const double *h;            /* [n] layer thickness [m] */
    const double *zc;           /* [n] depth of the layer centre [m] */
    const double *lat;          /* [ncol] latitude [degrees] */
    const int *rowptr;          /* [n+1] explicit matrices: CSR row pointers */
    const int *colidx;          /* [nnz] column indices */
    const double *exp_val;      /* [nmonth][nnz] values */
    const long long *blk_off;   /* [ncol+1] implicit matrices: offset of each column block */
    const double *imp_blk;      /* [nmonth][s_imp] dense row-major blocks */
    long long s_imp;
} oracle_problem;

/* ---------------------------------------------------------------------------------
 * Interpolation weights in time (Section 3; reading R3).
 * Step j starts at t_j = j / nstep (fraction of a year).  With monthly matrices at
 * mid-month, s = nmonth t_j - 1/2, m0 = floor(s) mod nmonth, m1 = m0 + 1 mod nmonth,
 * w = s - floor(s), and the operator is (1 - w) M_m0 + w M_m1.  s is formed from
 * integers, num / den with num = 2 nmonth j - nstep and den = 2 nstep, so that w is
 * exactly 0 on the month centres.
 * --------------------------------------------------------------------------------- */
void oracle_month_weights(int j, int nstep, int nmonth, int *m0, int *m1, double *w)
{
    long long num = 2LL * nmonth * j - nstep;
    long long den = 2LL * nstep;
    long long k = num / den;
    if (num % den != 0 && num < 0) k -= 1;          /* floor division */
    long long r = num - k * den;                    /* 0 <= r < den */
    int mk = (int)(((k % nmonth) + nmonth) % nmonth);
    *m0 = mk;
    *m1 = (mk + 1) % nmonth;
    *w = (double)r / (double)den;
}

/* ---------------------------------------------------------------------------------
 * Short-wave radiation I_SWR (Section 2.2.1 names Paltridge & Platt without giving the
 * formula; reading R8): daily-mean insolation at the top of the atmosphere,
 *   Q = S0/pi (h0 sin(phi) sin(delta) + cos(phi) cos(delta) sin(h0)),
 *   h0 = arccos(clamp(-tan(phi) tan(delta), -1, 1)),
 *   delta = -23.44 deg cos(2 pi (t + 10/360)),  S0 = 1361 W/m^2,
 * t the time as a fraction of the 360-day year.  *dayfrac = h0 / pi (daylight fraction).
 * --------------------------------------------------------------------------------- */
double oracle_insolation(double lat_deg, double t, double *dayfrac)
{
    const double pi = 3.14159265358979323846;
    const double S0 = 1361.0;
    double phi = lat_deg * (pi / 180.0);
    double delta = -23.44 * (pi / 180.0) * cos(2.0 * pi * (t + 10.0 / 360.0));
    double x = -tan(phi) * tan(delta);
    if (x > 1.0) x = 1.0;
    if (x < -1.0) x = -1.0;
    double h0 = acos(x);
    if (dayfrac) *dayfrac = h0 / pi;
    return S0 / pi * (h0 * sin(phi) * sin(delta) + cos(phi) * cos(delta) * sin(h0));
}

/* ---------------------------------------------------------------------------------
 * PO4-DOP source-minus-sink term (Section 2.2.1), one evaluation on one column.
 * Tracers: y1 = N (phosphate), y2 = DOP.  Parameters u, in this order:
 *   u[0] k_w   attenuation of water [1/m]           (K_H2O)
 *   u[1] alpha maximum community production [1/d]
 *   u[2] sigma fraction of production to DOP [-]     (sigma_2; sigma_bar = 1 - sigma)
 *   u[3] lambda DOP remineralisation rate [1/yr]     (lambda'_2)
 *   u[4] K_N   half saturation of PO4               (K_1)
 *   u[5] K_I   half saturation of light [W/m^2]
 *   u[6] b     Martin exponent [-]
 * Euphotic zone Omega_1: the top min(2, nlayer) layers (Section 7: two euphotic layers).
 *   I_k  = I_SWR sigma_PAR (1 - sigma_ice) exp(-d_k k_w)
 *   f_k  = alpha N_k/(N_k + K_N) I_k/(I_k + K_I)
 *   q1_k = -f_k + lambda DOP_k,   q2_k = sigma f_k - lambda DOP_k
 * Export through the base z_eu of the euphotic zone: E = (1 - sigma) sum_k f_k h_k,
 * flux F(z) = E (z / z_eu)^(-b)  (Martin et al.).
 * Aphotic zone Omega_2:
 *   q1_k = (F(z_top,k) - F(z_bot,k)) / h_k + lambda DOP_k,  q2_k = -lambda DOP_k
 * with F(z_bot) = 0 in the bottom layer (R5-R7).  Rates are per year (R9).
 * --------------------------------------------------------------------------------- */
static void ndop_q(int nlayer, const double *h, const double *d, double insol, double ice,
                   const double *N, const double *DOP, const double *u, double *qN, double *qD)
{
    const double sigma_par = 0.4;
    double kw = u[0], alpha = u[1] * 360.0, sigma = u[2], lambda = u[3];
    double KN = u[4], KI = u[5], b = u[6];
    int neu = nlayer < 2 ? nlayer : 2;
    double E = 0.0;
    double zeu = 0.0;
    for (int k = 0; k < neu; k++) {
        double I = insol * sigma_par * (1.0 - ice) * exp(-d[k] * kw);
        double f = alpha * (N[k] / (N[k] + KN)) * (I / (I + KI));
        qN[k] = -f + lambda * DOP[k];
        qD[k] = sigma * f - lambda * DOP[k];
        E += (1.0 - sigma) * f * h[k];
        zeu += h[k];
    }
    double ztop = zeu;
    for (int k = neu; k < nlayer; k++) {
        double zbot = ztop + h[k];
        double Ftop = E * pow(ztop / zeu, -b);
        double Fbot = (k == nlayer - 1) ? 0.0 : E * pow(zbot / zeu, -b);
        qN[k] = (Ftop - Fbot) / h[k] + lambda * DOP[k];
        qD[k] = -lambda * DOP[k];
        ztop = zbot;
    }
    if (nlayer <= neu)
        qN[nlayer - 1] += E / h[nlayer - 1];
}

/* ---------------------------------------------------------------------------------
 * N model (reading R10): PO4 alone, parameters u, in this order:
 *   u[0] k_w, u[1] alpha [1/d], u[2] K_N, u[3] K_I, u[4] b.
 * Euphotic layers: q_k = -f_k with f_k as in the PO4-DOP model; the whole production is
 * exported, E = sum_k f_k h_k, and remineralised below with Martin's law; the same bottom
 * rule as the PO4-DOP model.
 * --------------------------------------------------------------------------------- */
static void n_q(int nlayer, const double *h, const double *d, double insol, double ice,
                const double *PO4, const double *u, double *q)
{
    const double sigma_par = 0.4;
    double kw = u[0], alpha = 360.0 * u[1], KN = u[2], KI = u[3], b = u[4];
    int neu = nlayer < 2 ? nlayer : 2;
    double E = 0.0, zeu = 0.0;
    for (int k = 0; k < neu; k++) {
        double I = insol * sigma_par * (1.0 - ice) * exp(-kw * d[k]);
        double f = alpha * (PO4[k] / (PO4[k] + KN)) * (I / (KI + I));
        q[k] = -f;
        E += f * h[k];
        zeu += h[k];
    }
    double ztop = zeu;
    for (int k = neu; k < nlayer; k++) {
        double zbot = ztop + h[k];
        double top = pow(ztop / zeu, -b);
        double bot = (k + 1 < nlayer) ? pow(zbot / zeu, -b) : 0.0;
        q[k] = E * (top - bot) / h[k];
        ztop = zbot;
    }
    if (neu >= nlayer)
        q[nlayer - 1] += E / h[nlayer - 1];
}

/* ---------------------------------------------------------------------------------
 * PO4-DOP-PHY model (Section 2.2.2; reading R11).  Tracers y1 = PO4, y2 = DOP,
 * y3 = PHY.  Parameters u, in the order of the paper's table:
 *   u[0] mu_1 maximum growth [1/d]      u[1] K_H2O (k_w) [1/m]   u[2] K_1
 *   u[3] K_I [W/m^2]                    u[4] lambda'_2 DOP remineralisation [1/d]
 *   u[5] sigma_2                        u[6] lambda_3 PHY loss, euphotic [1/d]
 *   u[7] kappa_3 quadratic PHY loss [1/d per mmol P/m^3]
 *   u[8] lambda'_3 PHY loss, whole column [1/d]   u[9] sigma_3   u[10] b
 * Euphotic:  f_1 = mu_1 PHY PO4/(PO4 + K_1) I/(I + K_I),  f_3 = sigma_3 f_1,
 *   q1 = -f_1 + l2 DOP,
 *   q2 = sigma_2 f_3 + l3 PHY + k3 PHY^2 - l2 DOP + l3' PHY,
 *   q3 = (1 - sigma_3) f_1 - l3 PHY - k3 PHY^2 - l3' PHY,
 *   E  = (1 - sigma_2) sum_k f_3,k h_k.
 * Aphotic:   q1 = (F(z_top) - F(z_bot))/h + l2 DOP,  q2 = -l2 DOP + l3' PHY,
 *   q3 = -l3' PHY, with Martin's F and the bottom rule of the PO4-DOP model.
 * --------------------------------------------------------------------------------- */
static void phy_q(int nlayer, const double *h, const double *d, double insol, double ice,
                  const double *y, const double *u, double *q)
{
    const double sigma_par = 0.4;
    const double *PO4 = y, *DOP = y + nlayer, *PHY = y + 2 * nlayer;
    double *q1 = q, *q2 = q + nlayer, *q3 = q + 2 * nlayer;
    double mu1 = 360.0 * u[0], kw = u[1], K1 = u[2], KI = u[3], l2 = 360.0 * u[4];
    double sig2 = u[5], l3 = 360.0 * u[6], k3 = 360.0 * u[7], l3p = 360.0 * u[8];
    double sig3 = u[9], b = u[10];
    int neu = nlayer < 2 ? nlayer : 2;
    double E = 0.0, zeu = 0.0;
    for (int k = 0; k < neu; k++) {
        double I = insol * sigma_par * (1.0 - ice) * exp(-kw * d[k]);
        double f1 = mu1 * PHY[k] * (PO4[k] / (PO4[k] + K1)) * (I / (KI + I));
        double f3 = sig3 * f1;
        double loss = l3 * PHY[k] + k3 * PHY[k] * PHY[k];
        q1[k] = -f1 + l2 * DOP[k];
        q2[k] = sig2 * f3 + loss - l2 * DOP[k] + l3p * PHY[k];
        q3[k] = (1.0 - sig3) * f1 - loss - l3p * PHY[k];
        E += (1.0 - sig2) * f3 * h[k];
        zeu += h[k];
    }
    double ztop = zeu;
    for (int k = neu; k < nlayer; k++) {
        double zbot = ztop + h[k];
        double top = pow(ztop / zeu, -b);
        double bot = (k + 1 < nlayer) ? pow(zbot / zeu, -b) : 0.0;
        q1[k] = E * (top - bot) / h[k] + l2 * DOP[k];
        q2[k] = -l2 * DOP[k] + l3p * PHY[k];
        q3[k] = -l3p * PHY[k];
        ztop = zbot;
    }
    if (neu >= nlayer)
        q1[nlayer - 1] += E / h[nlayer - 1];
}

/* ---------------------------------------------------------------------------------
 * NPZD-DOP model (reading R12).  Tracers N (PO4), P (phytoplankton), Z (zooplankton),
 * D (detritus), DOP.  Parameters u, in this order:
 *   u[0] k_w [1/m]        u[1] mu_P max growth [1/d]   u[2] K_N     u[3] K_I [W/m^2]
 *   u[4] mu_Z max grazing [1/d]   u[5] K_P grazing half saturation   u[6] epsilon
 *   assimilated fraction of grazing   u[7] lambda_P P mortality [1/d]
 *   u[8] kappa_Z quadratic Z mortality [1/d per mmol P/m^3]   u[9] lambda_Z Z excretion
 *   [1/d]   u[10] lambda_D detritus remineralisation [1/d]   u[11] lambda_DOP DOP
 *   remineralisation [1/d]   u[12] w_D detritus sinking speed [m/d].
 * Rates per cell:
 *   U = mu_P P N/(N + K_N) I/(I + K_I)  (euphotic layers only),  G = mu_Z Z P/(K_P + P),
 *   and linear or quadratic losses lambda_P P, kappa_Z Z^2, lambda_Z Z, lambda_D D,
 *   lambda_DOP DOP.  Sinking: S_k = w_D D_k through the base of layer k, S = 0 through
 *   the sea floor and into the top layer.
 *   qN = -U + lambda_DOP DOP
 *   qP = U - G - lambda_P P
 *   qZ = epsilon G - kappa_Z Z^2 - lambda_Z Z
 *   qD = lambda_P P + kappa_Z Z^2 - lambda_D D + (S_{k-1} - S_k) / h_k
 *   qDOP = (1 - epsilon) G + lambda_Z Z + lambda_D D - lambda_DOP DOP
 * --------------------------------------------------------------------------------- */
static void npzd_q(int nlayer, const double *h, const double *d, double insol, double ice,
                   const double *y, const double *u, double *q)
{
    const double sigma_par = 0.4;
    const double *N = y, *P = y + nlayer, *Z = y + 2 * nlayer, *D = y + 3 * nlayer;
    const double *DOP = y + 4 * nlayer;
    double kw = u[0], muP = 360.0 * u[1], KN = u[2], KI = u[3], muZ = 360.0 * u[4];
    double KP = u[5], eps = u[6], lP = 360.0 * u[7], kZ = 360.0 * u[8], lZ = 360.0 * u[9];
    double lD = 360.0 * u[10], lO = 360.0 * u[11], wD = 360.0 * u[12];
    int neu = nlayer < 2 ? nlayer : 2;
    double Sin = 0.0;                       /* sinking flux into the top of layer k */
    for (int k = 0; k < nlayer; k++) {
        double U = 0.0;
        if (k < neu) {
            double I = insol * sigma_par * (1.0 - ice) * exp(-kw * d[k]);
            U = muP * P[k] * (N[k] / (N[k] + KN)) * (I / (KI + I));
        }
        double G = muZ * Z[k] * (P[k] / (KP + P[k]));
        double mP = lP * P[k], mZ = kZ * Z[k] * Z[k], eZ = lZ * Z[k];
        double rD = lD * D[k], rO = lO * DOP[k];
        double Sout = (k + 1 < nlayer) ? wD * D[k] : 0.0;
        q[k] = -U + rO;
        q[nlayer + k] = U - G - mP;
        q[2 * nlayer + k] = eps * G - mZ - eZ;
        q[3 * nlayer + k] = mP + mZ - rD + (Sin - Sout) / h[k];
        q[4 * nlayer + k] = (1.0 - eps) * G + eZ + rD - rO;
        Sin = Sout;
    }
}

/* q of one column for any model; y and q are (ntracer, nlayer), layer index fastest. */
static int model_q(int model, int ntracer, int nparam, int nlayer, const double *h,
                   const double *d, double insol, double ice, const double *y,
                   const double *u, double *q)
{
    if (model == ORACLE_MODEL_NDOP && ntracer == 2 && nparam == 7) {
        ndop_q(nlayer, h, d, insol, ice, y, y + nlayer, u, q, q + nlayer);
        return 0;
    }
    if (model == ORACLE_MODEL_N && ntracer == 1 && nparam == 5) {
        n_q(nlayer, h, d, insol, ice, y, u, q);
        return 0;
    }
    if (model == ORACLE_MODEL_PHY && ntracer == 3 && nparam == 11) {
        phy_q(nlayer, h, d, insol, ice, y, u, q);
        return 0;
    }
    if (model == ORACLE_MODEL_NPZD && ntracer == 5 && nparam == 13) {
        npzd_q(nlayer, h, d, insol, ice, y, u, q);
        return 0;
    }
    return -1;
}

/* ---------------------------------------------------------------------------------
 * The model interface of Section 5.2:
 *   bgc(t, dt, lat, insol, dayfrac, ice, wind, ntracer, nlayer, h, d, salt, temp,
 *       y, ybgc, nparam, u)
 * y and ybgc are (nlayer, ntracer) arrays with the layer index fastest.  ybgc receives
 * the increment over the ocean step dt (R1, R2): nsub explicit Euler steps of length
 * dt / nsub with the same forcing.  lat, dayfrac, wind, salt and temp are part of the
 * interface and unused by this model.  Returns 0, or -1 on bad arguments.
 * --------------------------------------------------------------------------------- */
int oracle_bgc(int model, double t, double dt, double lat, double insol, double dayfrac,
               double ice, double wind, int ntracer, int nlayer, const double *h,
               const double *d, const double *salt, const double *temp, const double *y,
               double *ybgc, int nparam, const double *u, int nsub)
{
    (void)t; (void)lat; (void)dayfrac; (void)wind; (void)salt; (void)temp;
    if (nlayer < 1 || nlayer > ORACLE_MAX_LAYER || nsub < 1) return -1;
    if (model == ORACLE_MODEL_NONE) {
        for (int i = 0; i < ntracer * nlayer; i++) ybgc[i] = 0.0;
        return 0;
    }
    if (ntracer < 1 || ntracer > ORACLE_MAX_TRACER) return -1;
    double ys[ORACLE_MAX_TRACER * ORACLE_MAX_LAYER], q[ORACLE_MAX_TRACER * ORACLE_MAX_LAYER];
    int len = ntracer * nlayer;
    memcpy(ys, y, sizeof(double) * len);
    double ds = dt / nsub;
    for (int s = 0; s < nsub; s++) {
        if (model_q(model, ntracer, nparam, nlayer, h, d, insol, ice, ys, u, q) != 0) return -1;
        for (int i = 0; i < len; i++) ys[i] += ds * q[i];
    }
    for (int i = 0; i < len; i++) ybgc[i] = ys[i] - y[i];
    return 0;
}

/* ---------------------------------------------------------------------------------
 * One TMM step (Section 3): y_out = A_imp(t_j) (A_exp(t_j) y + q_j(y, u)).
 * State layout [ntracer][n]; cells ordered column by column, surface to bottom.
 * work: caller-provided [ntracer][n] scratch.
 * --------------------------------------------------------------------------------- */
int oracle_step(const oracle_problem *P, int model, int ntracer, int j, const double *y,
                double *y_out, const double *u, int nparam, int nsub, double *work)
{
    int n = P->n;
    int m0, m1;
    double w;
    oracle_month_weights(j, P->nstep, P->nmonth, &m0, &m1, &w);
    double t = (double)j / P->nstep;
    double dt = 1.0 / P->nstep;
    const double *a0 = P->exp_val + (size_t)m0 * P->nnz;
    const double *a1 = P->exp_val + (size_t)m1 * P->nnz;
    const double *b0 = P->imp_blk + (size_t)m0 * P->s_imp;
    const double *b1 = P->imp_blk + (size_t)m1 * P->s_imp;
    double *z = work;
    int bad = 0;

    /* explicit part: z = A_exp(t_j) y, A_exp(t_j) = (1 - w) A_m0 + w A_m1 */
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        for (int tr = 0; tr < ntracer; tr++) {
            double s = 0.0;
            for (int p = P->rowptr[i]; p < P->rowptr[i + 1]; p++) {
                double a = (1.0 - w) * a0[p] + w * a1[p];
                s += a * y[(size_t)tr * n + P->colidx[p]];
            }
            z[(size_t)tr * n + i] = s;
        }
    }

    /* per column: add q(y_j), then the implicit part y_out = A_imp(t_j) z */
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int c = 0; c < P->ncol; c++) {
        int s0 = P->col_start[c];
        int L = P->col_start[c + 1] - s0;
        double ycol[ORACLE_MAX_LAYER * ORACLE_MAX_TRACER], dq[ORACLE_MAX_LAYER * ORACLE_MAX_TRACER];
        if (L > ORACLE_MAX_LAYER || ntracer > ORACLE_MAX_TRACER) { bad |= 1; continue; }
        for (int tr = 0; tr < ntracer; tr++)
            for (int k = 0; k < L; k++) ycol[tr * L + k] = y[(size_t)tr * n + s0 + k];
        double dayfrac;
        double insol = oracle_insolation(P->lat[c], t, &dayfrac);
        if (oracle_bgc(model, t, dt, P->lat[c], insol, dayfrac, 0.0, 0.0, ntracer, L,
                       P->h + s0, P->zc + s0, NULL, NULL, ycol, dq, nparam, u, nsub) != 0) {
            bad |= 1;
            continue;
        }
        for (int tr = 0; tr < ntracer; tr++)
            for (int k = 0; k < L; k++) z[(size_t)tr * n + s0 + k] += dq[tr * L + k];
        const double *B0 = b0 + P->blk_off[c];
        const double *B1 = b1 + P->blk_off[c];
        for (int tr = 0; tr < ntracer; tr++) {
            for (int r = 0; r < L; r++) {
                double s = 0.0;
                for (int k = 0; k < L; k++) {
                    double bb = (1.0 - w) * B0[r * L + k] + w * B1[r * L + k];
                    s += bb * z[(size_t)tr * n + s0 + k];
                }
                y_out[(size_t)tr * n + s0 + r] = s;
            }
        }
    }
    return bad ? -1 : 0;
}

/* ---------------------------------------------------------------------------------
 * The year map phi (Section 4): nstep steps from y0, result in y1.
 * --------------------------------------------------------------------------------- */
int oracle_year_map(const oracle_problem *P, int model, int ntracer, const double *y0,
                    double *y1, const double *u, int nparam, int nsub)
{
    size_t len = (size_t)ntracer * P->n;
    double *a = (double *)malloc(sizeof(double) * len);
    double *b = (double *)malloc(sizeof(double) * len);
    double *work = (double *)malloc(sizeof(double) * len);
    if (!a || !b || !work) { free(a); free(b); free(work); return -2; }
    memcpy(a, y0, sizeof(double) * len);
    int rc = 0;
    for (int j = 0; j < P->nstep && rc == 0; j++) {
        rc = oracle_step(P, model, ntracer, j, a, b, u, nparam, nsub, work);
        double *tmp = a; a = b; b = tmp;
    }
    memcpy(y1, a, sizeof(double) * len);
    free(a); free(b); free(work);
    return rc;
}

/* Run nsteps steps starting at step j0 (steps wrap around the year). */
int oracle_steps(const oracle_problem *P, int model, int ntracer, int j0, int nsteps,
                 const double *y0, double *y1, const double *u, int nparam, int nsub)
{
    size_t len = (size_t)ntracer * P->n;
    double *a = (double *)malloc(sizeof(double) * len);
    double *b = (double *)malloc(sizeof(double) * len);
    double *work = (double *)malloc(sizeof(double) * len);
    if (!a || !b || !work) { free(a); free(b); free(work); return -2; }
    memcpy(a, y0, sizeof(double) * len);
    int rc = 0;
    for (int s = 0; s < nsteps && rc == 0; s++) {
        rc = oracle_step(P, model, ntracer, (j0 + s) % P->nstep, a, b, u, nparam, nsub, work);
        double *tmp = a; a = b; b = tmp;
    }
    memcpy(y1, a, sizeof(double) * len);
    free(a); free(b); free(work);
    return rc;
}

/* Threads used by the OpenMP loops above (1 when built without OpenMP). */
int oracle_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* ---------------------------------------------------------------------------------
 * Tangent-linear model.  Section 6 names exact Jacobian-vector products (by algorithmic
 * differentiation) as the alternative to finite differences; here the derivative of the
 * PO4-DOP equations of Section 2.2.1 is written out by hand:
 *   df_k  = alpha K_N / (N_k + K_N)^2 I_k / (I_k + K_I) dN_k
 *   dq1_k = -df_k + lambda dDOP_k,   dq2_k = sigma df_k - lambda dDOP_k      (euphotic)
 *   dE    = (1 - sigma) sum_k df_k h_k,   dF(z) = dE (z / z_eu)^(-b)
 *   dq1_k = (dF(z_top) - dF(z_bot)) / h_k + lambda dDOP_k, dq2_k = -lambda dDOP_k (aphotic)
 * and each internal Euler step y <- y + ds q(y) has the tangent dy <- dy + ds dq(y; dy).
 * --------------------------------------------------------------------------------- */
static void ndop_q_tangent(int nlayer, const double *h, const double *d, double insol, double ice,
                           const double *N, const double *DOP, const double *dN, const double *dDOP,
                           const double *u, double *qN, double *qD, double *dqN, double *dqD)
{
    const double sigma_par = 0.4;
    double kw = u[0], alpha = u[1] * 360.0, sigma = u[2], lambda = u[3];
    double KN = u[4], KI = u[5], b = u[6];
    int neu = nlayer < 2 ? nlayer : 2;
    double E = 0.0, dE = 0.0, zeu = 0.0;
    for (int k = 0; k < neu; k++) {
        double I = insol * sigma_par * (1.0 - ice) * exp(-d[k] * kw);
        double LF = I / (I + KI);
        double f = alpha * (N[k] / (N[k] + KN)) * LF;
        double df = alpha * (KN / ((N[k] + KN) * (N[k] + KN))) * LF * dN[k];
        qN[k] = -f + lambda * DOP[k];
        qD[k] = sigma * f - lambda * DOP[k];
        dqN[k] = -df + lambda * dDOP[k];
        dqD[k] = sigma * df - lambda * dDOP[k];
        E += (1.0 - sigma) * f * h[k];
        dE += (1.0 - sigma) * df * h[k];
        zeu += h[k];
    }
    double ztop = zeu;
    for (int k = neu; k < nlayer; k++) {
        double zbot = ztop + h[k];
        double pt = pow(ztop / zeu, -b);
        double pb = (k == nlayer - 1) ? 0.0 : pow(zbot / zeu, -b);
        qN[k] = (E * pt - E * pb) / h[k] + lambda * DOP[k];
        qD[k] = -lambda * DOP[k];
        dqN[k] = (dE * pt - dE * pb) / h[k] + lambda * dDOP[k];
        dqD[k] = -lambda * dDOP[k];
        ztop = zbot;
    }
    if (nlayer <= neu) {
        qN[nlayer - 1] += E / h[nlayer - 1];
        dqN[nlayer - 1] += dE / h[nlayer - 1];
    }
}

/* Tangent of the N model (R10), by hand: df_k = alpha K_N / (PO4_k + K_N)^2 I_k/(I_k + K_I) dPO4_k,
 * dq_k = -df_k (euphotic), dE = sum_k df_k h_k, dq_k = dE (top_k - bot_k) / h_k (aphotic), and
 * the shallow column's bottom layer gets dE / h. */
static void n_q_tangent(int nlayer, const double *h, const double *d, double insol, double ice,
                        const double *PO4, const double *dPO4, const double *u, double *q, double *dq)
{
    const double sigma_par = 0.4;
    double kw = u[0], alpha = 360.0 * u[1], KN = u[2], KI = u[3], b = u[4];
    int neu = nlayer < 2 ? nlayer : 2;
    double E = 0.0, dE = 0.0, zeu = 0.0;
    for (int k = 0; k < neu; k++) {
        double I = insol * sigma_par * (1.0 - ice) * exp(-kw * d[k]);
        double LF = I / (KI + I);
        double f = alpha * (PO4[k] / (PO4[k] + KN)) * LF;
        double df = alpha * (KN / ((PO4[k] + KN) * (PO4[k] + KN))) * LF * dPO4[k];
        q[k] = -f;
        dq[k] = -df;
        E += f * h[k];
        dE += df * h[k];
        zeu += h[k];
    }
    double ztop = zeu;
    for (int k = neu; k < nlayer; k++) {
        double zbot = ztop + h[k];
        double top = pow(ztop / zeu, -b);
        double bot = (k + 1 < nlayer) ? pow(zbot / zeu, -b) : 0.0;
        q[k] = E * (top - bot) / h[k];
        dq[k] = dE * (top - bot) / h[k];
        ztop = zbot;
    }
    if (neu >= nlayer) {
        q[nlayer - 1] += E / h[nlayer - 1];
        dq[nlayer - 1] += dE / h[nlayer - 1];
    }
}

/* Tangent of the PO4-DOP-PHY model (Section 2.2.2, R11), by hand.  With M = PO4/(PO4+K_1) and
 * LF = I/(I+K_I): df_1 = mu_1 LF (M dPHY + PHY K_1/(PO4+K_1)^2 dPO4), df_3 = sigma_3 df_1,
 * dloss = (lambda_3 + 2 kappa_3 PHY) dPHY, and every q is linear in those and in DOP, PHY. */
static void phy_q_tangent(int nlayer, const double *h, const double *d, double insol, double ice,
                          const double *y, const double *dy, const double *u, double *q, double *dq)
{
    const double sigma_par = 0.4;
    const double *PO4 = y, *DOP = y + nlayer, *PHY = y + 2 * nlayer;
    const double *dPO4 = dy, *dDOP = dy + nlayer, *dPHY = dy + 2 * nlayer;
    double *q1 = q, *q2 = q + nlayer, *q3 = q + 2 * nlayer;
    double *dq1 = dq, *dq2 = dq + nlayer, *dq3 = dq + 2 * nlayer;
    double mu1 = 360.0 * u[0], kw = u[1], K1 = u[2], KI = u[3], l2 = 360.0 * u[4];
    double sig2 = u[5], l3 = 360.0 * u[6], k3 = 360.0 * u[7], l3p = 360.0 * u[8];
    double sig3 = u[9], b = u[10];
    int neu = nlayer < 2 ? nlayer : 2;
    double E = 0.0, dE = 0.0, zeu = 0.0;
    for (int k = 0; k < neu; k++) {
        double I = insol * sigma_par * (1.0 - ice) * exp(-kw * d[k]);
        double LF = I / (KI + I);
        double M = PO4[k] / (PO4[k] + K1);
        double dM = K1 / ((PO4[k] + K1) * (PO4[k] + K1)) * dPO4[k];
        double f1 = mu1 * PHY[k] * M * LF;
        double df1 = mu1 * LF * (dPHY[k] * M + PHY[k] * dM);
        double f3 = sig3 * f1, df3 = sig3 * df1;
        double loss = l3 * PHY[k] + k3 * PHY[k] * PHY[k];
        double dloss = (l3 + 2.0 * k3 * PHY[k]) * dPHY[k];
        q1[k] = -f1 + l2 * DOP[k];
        q2[k] = sig2 * f3 + loss - l2 * DOP[k] + l3p * PHY[k];
        q3[k] = (1.0 - sig3) * f1 - loss - l3p * PHY[k];
        dq1[k] = -df1 + l2 * dDOP[k];
        dq2[k] = sig2 * df3 + dloss - l2 * dDOP[k] + l3p * dPHY[k];
        dq3[k] = (1.0 - sig3) * df1 - dloss - l3p * dPHY[k];
        E += (1.0 - sig2) * f3 * h[k];
        dE += (1.0 - sig2) * df3 * h[k];
        zeu += h[k];
    }
    double ztop = zeu;
    for (int k = neu; k < nlayer; k++) {
        double zbot = ztop + h[k];
        double top = pow(ztop / zeu, -b);
        double bot = (k + 1 < nlayer) ? pow(zbot / zeu, -b) : 0.0;
        q1[k] = E * (top - bot) / h[k] + l2 * DOP[k];
        q2[k] = -l2 * DOP[k] + l3p * PHY[k];
        q3[k] = -l3p * PHY[k];
        dq1[k] = dE * (top - bot) / h[k] + l2 * dDOP[k];
        dq2[k] = -l2 * dDOP[k] + l3p * dPHY[k];
        dq3[k] = -l3p * dPHY[k];
        ztop = zbot;
    }
    if (neu >= nlayer) {
        q1[nlayer - 1] += E / h[nlayer - 1];
        dq1[nlayer - 1] += dE / h[nlayer - 1];
    }
}

/* Tangent of the NPZD-DOP model (R12), by hand: dU = mu_P LF (M dP + P K_N/(N+K_N)^2 dN),
 * dG = mu_Z (P/(K_P+P) dZ + Z K_P/(K_P+P)^2 dP), the losses' derivatives, and the sinking
 * fluxes dS_k = w_D dD_k (none through the floor). */
static void npzd_q_tangent(int nlayer, const double *h, const double *d, double insol, double ice,
                           const double *y, const double *dy, const double *u, double *q, double *dq)
{
    const double sigma_par = 0.4;
    const double *N = y, *P = y + nlayer, *Z = y + 2 * nlayer, *D = y + 3 * nlayer;
    const double *DOP = y + 4 * nlayer;
    const double *dN = dy, *dP = dy + nlayer, *dZ = dy + 2 * nlayer, *dD = dy + 3 * nlayer;
    const double *dDOP = dy + 4 * nlayer;
    double kw = u[0], muP = 360.0 * u[1], KN = u[2], KI = u[3], muZ = 360.0 * u[4];
    double KP = u[5], eps = u[6], lP = 360.0 * u[7], kZ = 360.0 * u[8], lZ = 360.0 * u[9];
    double lD = 360.0 * u[10], lO = 360.0 * u[11], wD = 360.0 * u[12];
    int neu = nlayer < 2 ? nlayer : 2;
    double Sin = 0.0, dSin = 0.0;
    for (int k = 0; k < nlayer; k++) {
        double U = 0.0, dU = 0.0;
        if (k < neu) {
            double I = insol * sigma_par * (1.0 - ice) * exp(-kw * d[k]);
            double LF = I / (KI + I);
            double M = N[k] / (N[k] + KN);
            U = muP * P[k] * M * LF;
            dU = muP * LF * (M * dP[k] + P[k] * (KN / ((N[k] + KN) * (N[k] + KN))) * dN[k]);
        }
        double R = P[k] / (KP + P[k]);
        double G = muZ * Z[k] * R;
        double dG = muZ * (R * dZ[k] + Z[k] * (KP / ((KP + P[k]) * (KP + P[k]))) * dP[k]);
        double mP = lP * P[k], mZ = kZ * Z[k] * Z[k], eZ = lZ * Z[k];
        double dmP = lP * dP[k], dmZ = 2.0 * kZ * Z[k] * dZ[k], deZ = lZ * dZ[k];
        double rD = lD * D[k], rO = lO * DOP[k], drD = lD * dD[k], drO = lO * dDOP[k];
        double Sout = (k + 1 < nlayer) ? wD * D[k] : 0.0;
        double dSout = (k + 1 < nlayer) ? wD * dD[k] : 0.0;
        q[k] = -U + rO;
        q[nlayer + k] = U - G - mP;
        q[2 * nlayer + k] = eps * G - mZ - eZ;
        q[3 * nlayer + k] = mP + mZ - rD + (Sin - Sout) / h[k];
        q[4 * nlayer + k] = (1.0 - eps) * G + eZ + rD - rO;
        dq[k] = -dU + drO;
        dq[nlayer + k] = dU - dG - dmP;
        dq[2 * nlayer + k] = eps * dG - dmZ - deZ;
        dq[3 * nlayer + k] = dmP + dmZ - drD + (dSin - dSout) / h[k];
        dq[4 * nlayer + k] = (1.0 - eps) * dG + deZ + drD - drO;
        Sin = Sout;
        dSin = dSout;
    }
}

/* q and its tangent along dy for any model; y, dy, q, dq are (ntracer, nlayer). */
static int model_q_tangent(int model, int ntracer, int nparam, int nlayer, const double *h, const double *d,
                           double insol, double ice, const double *y, const double *dy, const double *u,
                           double *q, double *dq)
{
    if (model == ORACLE_MODEL_NDOP && ntracer == 2 && nparam == 7) {
        ndop_q_tangent(nlayer, h, d, insol, ice, y, y + nlayer, dy, dy + nlayer, u, q, q + nlayer, dq,
                       dq + nlayer);
        return 0;
    }
    if (model == ORACLE_MODEL_N && ntracer == 1 && nparam == 5) {
        n_q_tangent(nlayer, h, d, insol, ice, y, dy, u, q, dq);
        return 0;
    }
    if (model == ORACLE_MODEL_PHY && ntracer == 3 && nparam == 11) {
        phy_q_tangent(nlayer, h, d, insol, ice, y, dy, u, q, dq);
        return 0;
    }
    if (model == ORACLE_MODEL_NPZD && ntracer == 5 && nparam == 13) {
        npzd_q_tangent(nlayer, h, d, insol, ice, y, dy, u, q, dq);
        return 0;
    }
    return -1;
}

/* The model interface and its tangent: ybgc as oracle_bgc, dybgc its derivative along dy. */
int oracle_bgc_tangent(int model, double t, double dt, double lat, double insol, double dayfrac,
                       double ice, double wind, int ntracer, int nlayer, const double *h,
                       const double *d, const double *y, const double *dy, double *ybgc,
                       double *dybgc, int nparam, const double *u, int nsub)
{
    (void)t; (void)lat; (void)dayfrac; (void)wind;
    if (nlayer < 1 || nlayer > ORACLE_MAX_LAYER || nsub < 1) return -1;
    if (model == ORACLE_MODEL_NONE) {
        for (int i = 0; i < ntracer * nlayer; i++) { ybgc[i] = 0.0; dybgc[i] = 0.0; }
        return 0;
    }
    if (ntracer < 1 || ntracer > ORACLE_MAX_TRACER) return -1;
    int len = ntracer * nlayer;
    double ys[ORACLE_MAX_TRACER * ORACLE_MAX_LAYER], dys[ORACLE_MAX_TRACER * ORACLE_MAX_LAYER];
    double q[ORACLE_MAX_TRACER * ORACLE_MAX_LAYER], dq[ORACLE_MAX_TRACER * ORACLE_MAX_LAYER];
    memcpy(ys, y, sizeof(double) * len);
    memcpy(dys, dy, sizeof(double) * len);
    double ds = dt / nsub;
    for (int s = 0; s < nsub; s++) {
        if (model_q_tangent(model, ntracer, nparam, nlayer, h, d, insol, ice, ys, dys, u, q, dq) != 0) return -1;
        for (int i = 0; i < len; i++) {
            ys[i] += ds * q[i];
            dys[i] += ds * dq[i];
        }
    }
    for (int i = 0; i < len; i++) {
        ybgc[i] = ys[i] - y[i];
        dybgc[i] = dys[i] - dy[i];
    }
    return 0;
}

/* One TMM step and its tangent: y_out as oracle_step, dy_out = A_imp (A_exp dy + dq). */
int oracle_step_tangent(const oracle_problem *P, int model, int ntracer, int j, const double *y,
                        const double *dy, double *y_out, double *dy_out, const double *u, int nparam,
                        int nsub, double *work, double *dwork)
{
    int n = P->n;
    int m0, m1;
    double w;
    oracle_month_weights(j, P->nstep, P->nmonth, &m0, &m1, &w);
    double t = (double)j / P->nstep;
    double dt = 1.0 / P->nstep;
    const double *a0 = P->exp_val + (size_t)m0 * P->nnz;
    const double *a1 = P->exp_val + (size_t)m1 * P->nnz;
    const double *b0 = P->imp_blk + (size_t)m0 * P->s_imp;
    const double *b1 = P->imp_blk + (size_t)m1 * P->s_imp;
    double *z = work, *dz = dwork;
    int bad = 0;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        for (int tr = 0; tr < ntracer; tr++) {
            double s = 0.0, ds = 0.0;
            for (int p = P->rowptr[i]; p < P->rowptr[i + 1]; p++) {
                double a = (1.0 - w) * a0[p] + w * a1[p];
                s += a * y[(size_t)tr * n + P->colidx[p]];
                ds += a * dy[(size_t)tr * n + P->colidx[p]];
            }
            z[(size_t)tr * n + i] = s;
            dz[(size_t)tr * n + i] = ds;
        }
    }
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int c = 0; c < P->ncol; c++) {
        int s0 = P->col_start[c];
        int L = P->col_start[c + 1] - s0;
        double ycol[ORACLE_MAX_LAYER * ORACLE_MAX_TRACER], dycol[ORACLE_MAX_LAYER * ORACLE_MAX_TRACER];
        double dq[ORACLE_MAX_LAYER * ORACLE_MAX_TRACER], ddq[ORACLE_MAX_LAYER * ORACLE_MAX_TRACER];
        if (L > ORACLE_MAX_LAYER || ntracer > ORACLE_MAX_TRACER) { bad |= 1; continue; }
        for (int tr = 0; tr < ntracer; tr++)
            for (int k = 0; k < L; k++) {
                ycol[tr * L + k] = y[(size_t)tr * n + s0 + k];
                dycol[tr * L + k] = dy[(size_t)tr * n + s0 + k];
            }
        double dayfrac;
        double insol = oracle_insolation(P->lat[c], t, &dayfrac);
        if (oracle_bgc_tangent(model, t, dt, P->lat[c], insol, dayfrac, 0.0, 0.0, ntracer, L, P->h + s0,
                               P->zc + s0, ycol, dycol, dq, ddq, nparam, u, nsub) != 0) {
            bad |= 1;
            continue;
        }
        for (int tr = 0; tr < ntracer; tr++)
            for (int k = 0; k < L; k++) {
                z[(size_t)tr * n + s0 + k] += dq[tr * L + k];
                dz[(size_t)tr * n + s0 + k] += ddq[tr * L + k];
            }
        const double *B0 = b0 + P->blk_off[c];
        const double *B1 = b1 + P->blk_off[c];
        for (int tr = 0; tr < ntracer; tr++) {
            for (int r = 0; r < L; r++) {
                double s = 0.0, ds = 0.0;
                for (int k = 0; k < L; k++) {
                    double bb = (1.0 - w) * B0[r * L + k] + w * B1[r * L + k];
                    s += bb * z[(size_t)tr * n + s0 + k];
                    ds += bb * dz[(size_t)tr * n + s0 + k];
                }
                y_out[(size_t)tr * n + s0 + r] = s;
                dy_out[(size_t)tr * n + s0 + r] = ds;
            }
        }
    }
    return bad ? -1 : 0;
}

/* The year map and its tangent: y1 = phi(y0), dy1 = phi'(y0) dy0. */
int oracle_year_tangent(const oracle_problem *P, int model, int ntracer, const double *y0,
                        const double *dy0, double *y1, double *dy1, const double *u, int nparam, int nsub)
{
    size_t len = (size_t)ntracer * P->n;
    double *a = (double *)malloc(sizeof(double) * len), *b = (double *)malloc(sizeof(double) * len);
    double *da = (double *)malloc(sizeof(double) * len), *db = (double *)malloc(sizeof(double) * len);
    double *w1 = (double *)malloc(sizeof(double) * len), *w2 = (double *)malloc(sizeof(double) * len);
    int rc = (a && b && da && db && w1 && w2) ? 0 : -2;
    if (rc == 0) {
        memcpy(a, y0, sizeof(double) * len);
        memcpy(da, dy0, sizeof(double) * len);
        for (int j = 0; j < P->nstep && rc == 0; j++) {
            rc = oracle_step_tangent(P, model, ntracer, j, a, da, b, db, u, nparam, nsub, w1, w2);
            double *t1 = a; a = b; b = t1;
            double *t2 = da; da = db; db = t2;
        }
        memcpy(y1, a, sizeof(double) * len);
        memcpy(dy1, da, sizeof(double) * len);
    }
    free(a); free(b); free(da); free(db); free(w1); free(w2);
    return rc;
}

/* ---------------------------------------------------------------------------------
 * Adjoint model (reverse mode), for gradients with respect to the state and to the model
 * parameters u (the parameter optimisation named in Sections 1 and 9).  For one step
 * y_{j+1} = B (A y_j + dq(y_j, u)) and a cotangent ybar_{j+1}:
 *   zbar = B^T ybar_{j+1},  ybar_j = A^T zbar + (d dq / dy)^T zbar,  ubar += (d dq / du)^T zbar.
 * dq is the increment of nsub explicit Euler steps; its reverse runs the internal steps
 * backwards: ybar^(s) = ybar^(s+1) + ds (dq/dy)^T ybar^(s+1), ubar += ds (dq/du)^T ybar^(s+1).
 * --------------------------------------------------------------------------------- */

/* Reverse of one evaluation of the PO4-DOP q at (N, DOP): given cotangents qbN, qbD of
 * (qN, qD), add the cotangents of N, DOP into Nb, Db and of u into ub. */
static void ndop_q_adjoint(int nlayer, const double *h, const double *d, double insol, double ice,
                           const double *N, const double *DOP, const double *u, const double *qbN,
                           const double *qbD, double *Nb, double *Db, double *ub)
{
    const double sigma_par = 0.4;
    double kw = u[0], alpha = u[1] * 360.0, sigma = u[2], lambda = u[3];
    double KN = u[4], KI = u[5], b = u[6];
    int neu = nlayer < 2 ? nlayer : 2;
    double f[ORACLE_MAX_LAYER], I[ORACLE_MAX_LAYER];
    double E = 0.0, zeu = 0.0, sumfh = 0.0;
    for (int k = 0; k < neu; k++) {
        I[k] = insol * sigma_par * (1.0 - ice) * exp(-d[k] * kw);
        f[k] = alpha * (N[k] / (N[k] + KN)) * (I[k] / (I[k] + KI));
        sumfh += f[k] * h[k];
        zeu += h[k];
    }
    E = (1.0 - sigma) * sumfh;
    /* aphotic layers and the bottom deposit: contributions to Ebar, DOP, lambda, b */
    double Eb = 0.0;
    double ztop = zeu;
    for (int k = neu; k < nlayer; k++) {
        double zbot = ztop + h[k];
        double pt = pow(ztop / zeu, -b);
        double pb = (k == nlayer - 1) ? 0.0 : pow(zbot / zeu, -b);
        double dpt = -log(ztop / zeu) * pt;            /* d pt / d b */
        double dpb = (k == nlayer - 1) ? 0.0 : -log(zbot / zeu) * pb;
        Eb += qbN[k] * (pt - pb) / h[k];
        ub[6] += qbN[k] * E * (dpt - dpb) / h[k];
        Db[k] += lambda * (qbN[k] - qbD[k]);
        ub[3] += (qbN[k] - qbD[k]) * DOP[k];
        ztop = zbot;
    }
    if (nlayer <= neu) Eb += qbN[nlayer - 1] / h[nlayer - 1];
    /* E = (1 - sigma) sum f_k h_k */
    ub[2] += -Eb * sumfh;
    for (int k = 0; k < neu; k++) {
        double fb = Eb * (1.0 - sigma) * h[k] - qbN[k] + sigma * qbD[k];
        ub[2] += qbD[k] * f[k];
        Db[k] += lambda * (qbN[k] - qbD[k]);
        ub[3] += (qbN[k] - qbD[k]) * DOP[k];
        /* f = alpha' N/(N+KN) I/(I+KI), alpha' = 360 alpha, I = I_s exp(-d kw) */
        double M = N[k] / (N[k] + KN), LF = I[k] / (I[k] + KI);
        ub[1] += fb * 360.0 * M * LF;
        Nb[k] += fb * alpha * LF * KN / ((N[k] + KN) * (N[k] + KN));
        ub[4] += fb * alpha * LF * (-N[k] / ((N[k] + KN) * (N[k] + KN)));
        ub[5] += fb * alpha * M * (-I[k] / ((I[k] + KI) * (I[k] + KI)));
        ub[0] += fb * alpha * M * (KI / ((I[k] + KI) * (I[k] + KI))) * (-d[k] * I[k]);
    }
}

/* Reverse of the N model q (R10) at PO4, by hand: given the cotangent qb of q, add the
 * cotangent of PO4 into yb and of u into ub. */
static void n_q_adjoint(int nlayer, const double *h, const double *d, double insol, double ice,
                        const double *PO4, const double *u, const double *qb, double *yb, double *ub)
{
    const double sigma_par = 0.4;
    double kw = u[0], alpha = 360.0 * u[1], KN = u[2], KI = u[3], b = u[4];
    int neu = nlayer < 2 ? nlayer : 2;
    double I[ORACLE_MAX_LAYER], f[ORACLE_MAX_LAYER];
    double E = 0.0, zeu = 0.0;
    for (int k = 0; k < neu; k++) {
        I[k] = insol * sigma_par * (1.0 - ice) * exp(-kw * d[k]);
        f[k] = alpha * (PO4[k] / (PO4[k] + KN)) * (I[k] / (KI + I[k]));
        E += f[k] * h[k];
        zeu += h[k];
    }
    /* aphotic q_k = E (top - bot) / h_k; shallow bottom layer q += E / h */
    double Eb = 0.0, ztop = zeu;
    for (int k = neu; k < nlayer; k++) {
        double zbot = ztop + h[k];
        double top = pow(ztop / zeu, -b);
        double bot = (k + 1 < nlayer) ? pow(zbot / zeu, -b) : 0.0;
        double dtop = -log(ztop / zeu) * top;          /* d top / d b */
        double dbot = (k + 1 < nlayer) ? -log(zbot / zeu) * bot : 0.0;
        Eb += qb[k] * (top - bot) / h[k];
        ub[4] += qb[k] * E * (dtop - dbot) / h[k];
        ztop = zbot;
    }
    if (neu >= nlayer) Eb += qb[nlayer - 1] / h[nlayer - 1];
    /* euphotic q_k = -f_k, E = sum f_k h_k, f = alpha' M LF */
    for (int k = 0; k < neu; k++) {
        double fb = -qb[k] + Eb * h[k];
        double M = PO4[k] / (PO4[k] + KN), LF = I[k] / (KI + I[k]);
        ub[1] += fb * 360.0 * M * LF;
        yb[k] += fb * alpha * LF * KN / ((PO4[k] + KN) * (PO4[k] + KN));
        ub[2] += fb * alpha * LF * (-PO4[k] / ((PO4[k] + KN) * (PO4[k] + KN)));
        ub[3] += fb * alpha * M * (-I[k] / ((KI + I[k]) * (KI + I[k])));
        ub[0] += fb * alpha * M * (KI / ((KI + I[k]) * (KI + I[k]))) * (-d[k] * I[k]);
    }
}

/* Reverse of the PO4-DOP-PHY q (Section 2.2.2, R11) at y = (PO4, DOP, PHY), by hand. */
static void phy_q_adjoint(int nlayer, const double *h, const double *d, double insol, double ice,
                          const double *y, const double *u, const double *qb, double *yb, double *ub)
{
    const double sigma_par = 0.4;
    const double *PO4 = y, *DOP = y + nlayer, *PHY = y + 2 * nlayer;
    const double *qb1 = qb, *qb2 = qb + nlayer, *qb3 = qb + 2 * nlayer;
    double *PO4b = yb, *DOPb = yb + nlayer, *PHYb = yb + 2 * nlayer;
    double mu1 = 360.0 * u[0], kw = u[1], K1 = u[2], KI = u[3], l2 = 360.0 * u[4];
    double sig2 = u[5], l3 = 360.0 * u[6], k3 = 360.0 * u[7], l3p = 360.0 * u[8];
    double sig3 = u[9], b = u[10];
    int neu = nlayer < 2 ? nlayer : 2;
    double I[ORACLE_MAX_LAYER], f1[ORACLE_MAX_LAYER];
    double sumf3h = 0.0, zeu = 0.0;
    for (int k = 0; k < neu; k++) {
        I[k] = insol * sigma_par * (1.0 - ice) * exp(-kw * d[k]);
        f1[k] = mu1 * PHY[k] * (PO4[k] / (PO4[k] + K1)) * (I[k] / (KI + I[k]));
        sumf3h += sig3 * f1[k] * h[k];
        zeu += h[k];
    }
    double E = (1.0 - sig2) * sumf3h;
    /* aphotic: q1 = E (top - bot)/h + l2 DOP, q2 = -l2 DOP + l3' PHY, q3 = -l3' PHY */
    double Eb = 0.0, ztop = zeu;
    for (int k = neu; k < nlayer; k++) {
        double zbot = ztop + h[k];
        double top = pow(ztop / zeu, -b);
        double bot = (k + 1 < nlayer) ? pow(zbot / zeu, -b) : 0.0;
        double dtop = -log(ztop / zeu) * top;
        double dbot = (k + 1 < nlayer) ? -log(zbot / zeu) * bot : 0.0;
        Eb += qb1[k] * (top - bot) / h[k];
        ub[10] += qb1[k] * E * (dtop - dbot) / h[k];
        DOPb[k] += l2 * (qb1[k] - qb2[k]);
        ub[4] += 360.0 * (qb1[k] - qb2[k]) * DOP[k];
        PHYb[k] += l3p * (qb2[k] - qb3[k]);
        ub[8] += 360.0 * (qb2[k] - qb3[k]) * PHY[k];
        ztop = zbot;
    }
    if (neu >= nlayer) Eb += qb1[nlayer - 1] / h[nlayer - 1];
    /* E = (1 - sigma_2) sum f_3 h */
    ub[5] += -Eb * sumf3h;
    for (int k = 0; k < neu; k++) {
        double f3 = sig3 * f1[k];
        /* q2 = sigma_2 f3 + ..., E: f3b; f3 = sigma_3 f1 */
        double f3b = sig2 * qb2[k] + Eb * (1.0 - sig2) * h[k];
        ub[5] += qb2[k] * f3;
        double f1b = -qb1[k] + (1.0 - sig3) * qb3[k] + sig3 * f3b;
        ub[9] += f3b * f1[k] - qb3[k] * f1[k];
        /* loss = l3 PHY + k3 PHY^2 in q2 (+) and q3 (-) */
        double lossb = qb2[k] - qb3[k];
        PHYb[k] += lossb * (l3 + 2.0 * k3 * PHY[k]);
        ub[6] += 360.0 * lossb * PHY[k];
        ub[7] += 360.0 * lossb * PHY[k] * PHY[k];
        DOPb[k] += l2 * (qb1[k] - qb2[k]);
        ub[4] += 360.0 * (qb1[k] - qb2[k]) * DOP[k];
        PHYb[k] += l3p * (qb2[k] - qb3[k]);
        ub[8] += 360.0 * (qb2[k] - qb3[k]) * PHY[k];
        /* f1 = mu1 PHY M LF */
        double M = PO4[k] / (PO4[k] + K1), LF = I[k] / (KI + I[k]);
        ub[0] += f1b * 360.0 * PHY[k] * M * LF;
        PHYb[k] += f1b * mu1 * M * LF;
        PO4b[k] += f1b * mu1 * PHY[k] * LF * K1 / ((PO4[k] + K1) * (PO4[k] + K1));
        ub[2] += f1b * mu1 * PHY[k] * LF * (-PO4[k] / ((PO4[k] + K1) * (PO4[k] + K1)));
        ub[3] += f1b * mu1 * PHY[k] * M * (-I[k] / ((KI + I[k]) * (KI + I[k])));
        ub[1] += f1b * mu1 * PHY[k] * M * (KI / ((KI + I[k]) * (KI + I[k]))) * (-d[k] * I[k]);
    }
}

/* Reverse of the NPZD-DOP q (R12) at y = (N, P, Z, D, DOP), by hand. */
static void npzd_q_adjoint(int nlayer, const double *h, const double *d, double insol, double ice,
                           const double *y, const double *u, const double *qb, double *yb, double *ub)
{
    const double sigma_par = 0.4;
    const double *N = y, *P = y + nlayer, *Z = y + 2 * nlayer, *D = y + 3 * nlayer;
    const double *DOP = y + 4 * nlayer;
    const double *qbN = qb, *qbP = qb + nlayer, *qbZ = qb + 2 * nlayer, *qbD = qb + 3 * nlayer;
    const double *qbO = qb + 4 * nlayer;
    double *Nb = yb, *Pb = yb + nlayer, *Zb = yb + 2 * nlayer, *Db = yb + 3 * nlayer, *Ob = yb + 4 * nlayer;
    double kw = u[0], muP = 360.0 * u[1], KN = u[2], KI = u[3], muZ = 360.0 * u[4];
    double KP = u[5], eps = u[6], lP = 360.0 * u[7], kZ = 360.0 * u[8], lZ = 360.0 * u[9];
    double lD = 360.0 * u[10], lO = 360.0 * u[11], wD = 360.0 * u[12];
    int neu = nlayer < 2 ? nlayer : 2;
    for (int k = 0; k < nlayer; k++) {
        /* sinking: S_k = w_D D_k (k + 1 < nlayer) leaves layer k and enters layer k + 1 */
        if (k + 1 < nlayer) {
            double Sb = -qbD[k] / h[k] + qbD[k + 1] / h[k + 1];
            Db[k] += wD * Sb;
            ub[12] += 360.0 * D[k] * Sb;
        }
        /* linear and quadratic losses */
        double mPb = -qbP[k] + qbD[k];
        Pb[k] += lP * mPb;
        ub[7] += 360.0 * mPb * P[k];
        double mZb = -qbZ[k] + qbD[k];
        Zb[k] += 2.0 * kZ * Z[k] * mZb;
        ub[8] += 360.0 * mZb * Z[k] * Z[k];
        double eZb = -qbZ[k] + qbO[k];
        Zb[k] += lZ * eZb;
        ub[9] += 360.0 * eZb * Z[k];
        double rDb = -qbD[k] + qbO[k];
        Db[k] += lD * rDb;
        ub[10] += 360.0 * rDb * D[k];
        double rOb = qbN[k] - qbO[k];
        Ob[k] += lO * rOb;
        ub[11] += 360.0 * rOb * DOP[k];
        /* grazing G = mu_Z Z P/(K_P + P), assimilated fraction epsilon */
        double R = P[k] / (KP + P[k]);
        double G = muZ * Z[k] * R;
        double Gb = -qbP[k] + eps * qbZ[k] + (1.0 - eps) * qbO[k];
        ub[6] += G * (qbZ[k] - qbO[k]);
        Zb[k] += Gb * muZ * R;
        Pb[k] += Gb * muZ * Z[k] * KP / ((KP + P[k]) * (KP + P[k]));
        ub[4] += Gb * 360.0 * Z[k] * R;
        ub[5] += Gb * muZ * Z[k] * (-P[k] / ((KP + P[k]) * (KP + P[k])));
        /* uptake U = mu_P P M LF in the euphotic layers */
        if (k < neu) {
            double I = insol * sigma_par * (1.0 - ice) * exp(-kw * d[k]);
            double LF = I / (KI + I), M = N[k] / (N[k] + KN);
            double Ub = -qbN[k] + qbP[k];
            Pb[k] += Ub * muP * M * LF;
            Nb[k] += Ub * muP * P[k] * LF * KN / ((N[k] + KN) * (N[k] + KN));
            ub[1] += Ub * 360.0 * P[k] * M * LF;
            ub[2] += Ub * muP * P[k] * LF * (-N[k] / ((N[k] + KN) * (N[k] + KN)));
            ub[3] += Ub * muP * P[k] * M * (-I / ((KI + I) * (KI + I)));
            ub[0] += Ub * muP * P[k] * M * (KI / ((KI + I) * (KI + I))) * (-d[k] * I);
        }
    }
}

/* Reverse of q for any model: cotangent qb of q (ntracer, nlayer) at y; yb, ub accumulated. */
static int model_q_adjoint(int model, int ntracer, int nparam, int nlayer, const double *h, const double *d,
                           double insol, double ice, const double *y, const double *u, const double *qb, double *yb,
                           double *ub)
{
    if (model == ORACLE_MODEL_NDOP && ntracer == 2 && nparam == 7) {
        ndop_q_adjoint(nlayer, h, d, insol, ice, y, y + nlayer, u, qb, qb + nlayer, yb, yb + nlayer, ub);
        return 0;
    }
    if (model == ORACLE_MODEL_N && ntracer == 1 && nparam == 5) {
        n_q_adjoint(nlayer, h, d, insol, ice, y, u, qb, yb, ub);
        return 0;
    }
    if (model == ORACLE_MODEL_PHY && ntracer == 3 && nparam == 11) {
        phy_q_adjoint(nlayer, h, d, insol, ice, y, u, qb, yb, ub);
        return 0;
    }
    if (model == ORACLE_MODEL_NPZD && ntracer == 5 && nparam == 13) {
        npzd_q_adjoint(nlayer, h, d, insol, ice, y, u, qb, yb, ub);
        return 0;
    }
    return -1;
}

/* Reverse of the model interface: given ybgc_bar (cotangent of ybgc), add the cotangent of
 * y into ybar and of u into ubar (both accumulated). */
int oracle_bgc_adjoint(int model, double dt, double insol, double ice, int ntracer, int nlayer,
                       const double *h, const double *d, const double *y, const double *ybgc_bar,
                       double *ybar, int nparam, const double *u, double *ubar, int nsub)
{
    if (nlayer < 1 || nlayer > ORACLE_MAX_LAYER || nsub < 1 || nsub > 64) return -1;
    if (model == ORACLE_MODEL_NONE) return 0;
    if (ntracer < 1 || ntracer > ORACLE_MAX_TRACER) return -1;
    int len = ntracer * nlayer;
    /* forward internal states y^(0..nsub-1) */
    static __thread double st[64][ORACLE_MAX_TRACER * ORACLE_MAX_LAYER];
    double q[ORACLE_MAX_TRACER * ORACLE_MAX_LAYER];
    double ds = dt / nsub;
    memcpy(st[0], y, sizeof(double) * len);
    for (int s = 0; s + 1 < nsub; s++) {
        if (model_q(model, ntracer, nparam, nlayer, h, d, insol, ice, st[s], u, q) != 0) return -1;
        for (int i = 0; i < len; i++) st[s + 1][i] = st[s][i] + ds * q[i];
    }
    /* ybgc = y^(nsub) - y^(0): ybar^(nsub) = ybgc_bar, and -ybgc_bar goes to y^(0); each
     * internal step y^(s+1) = y^(s) + ds q(y^(s)) passes ybar^(s) = ybar^(s+1) + (ds dq/dy)^T ybar^(s+1) */
    double yb[ORACLE_MAX_TRACER * ORACLE_MAX_LAYER], qb[ORACLE_MAX_TRACER * ORACLE_MAX_LAYER];
    memcpy(yb, ybgc_bar, sizeof(double) * len);
    for (int s = nsub - 1; s >= 0; s--) {
        for (int i = 0; i < len; i++) qb[i] = ds * yb[i];
        if (model_q_adjoint(model, ntracer, nparam, nlayer, h, d, insol, ice, st[s], u, qb, yb, ubar) != 0) return -1;
    }
    for (int i = 0; i < len; i++) ybar[i] += yb[i] - ybgc_bar[i];
    return 0;
}

/* Reverse of one TMM step at state y (step j): ybar_in = cotangent of y_{j+1};
 * ybar_out = cotangent of y_j; ubar accumulated.  work: [ntracer][n] scratch. */
int oracle_step_adjoint(const oracle_problem *P, int model, int ntracer, int j, const double *y,
                        const double *ybar_in, double *ybar_out, const double *u, int nparam,
                        double *ubar, int nsub, double *zbar)
{
    int n = P->n;
    int m0, m1;
    double w;
    oracle_month_weights(j, P->nstep, P->nmonth, &m0, &m1, &w);
    double t = (double)j / P->nstep;
    double dt = 1.0 / P->nstep;
    const double *a0 = P->exp_val + (size_t)m0 * P->nnz;
    const double *a1 = P->exp_val + (size_t)m1 * P->nnz;
    const double *b0 = P->imp_blk + (size_t)m0 * P->s_imp;
    const double *b1 = P->imp_blk + (size_t)m1 * P->s_imp;
    /* zbar = B^T ybar_in */
    for (int c = 0; c < P->ncol; c++) {
        int s0 = P->col_start[c], L = P->col_start[c + 1] - s0;
        const double *B0 = b0 + P->blk_off[c], *B1 = b1 + P->blk_off[c];
        for (int tr = 0; tr < ntracer; tr++)
            for (int k = 0; k < L; k++) {
                double s = 0.0;
                for (int r = 0; r < L; r++) {
                    double bb = (1.0 - w) * B0[r * L + k] + w * B1[r * L + k];
                    s += bb * ybar_in[(size_t)tr * n + s0 + r];
                }
                zbar[(size_t)tr * n + s0 + k] = s;
            }
    }
    /* ybar_out = A^T zbar */
    for (size_t i = 0; i < (size_t)ntracer * n; i++) ybar_out[i] = 0.0;
    for (int i = 0; i < n; i++)
        for (int p = P->rowptr[i]; p < P->rowptr[i + 1]; p++) {
            double a = (1.0 - w) * a0[p] + w * a1[p];
            for (int tr = 0; tr < ntracer; tr++)
                ybar_out[(size_t)tr * n + P->colidx[p]] += a * zbar[(size_t)tr * n + i];
        }
    /* + (d dq/dy)^T zbar, ubar += (d dq/du)^T zbar, column by column */
    for (int c = 0; c < P->ncol; c++) {
        int s0 = P->col_start[c], L = P->col_start[c + 1] - s0;
        double ycol[ORACLE_MAX_LAYER * ORACLE_MAX_TRACER], zb[ORACLE_MAX_LAYER * ORACLE_MAX_TRACER];
        double yb[ORACLE_MAX_LAYER * ORACLE_MAX_TRACER];
        if (L > ORACLE_MAX_LAYER || ntracer > ORACLE_MAX_TRACER) return -1;
        for (int tr = 0; tr < ntracer; tr++)
            for (int k = 0; k < L; k++) {
                ycol[tr * L + k] = y[(size_t)tr * n + s0 + k];
                zb[tr * L + k] = zbar[(size_t)tr * n + s0 + k];
                yb[tr * L + k] = 0.0;
            }
        double dayfrac;
        double insol = oracle_insolation(P->lat[c], t, &dayfrac);
        if (oracle_bgc_adjoint(model, dt, insol, 0.0, ntracer, L, P->h + s0, P->zc + s0, ycol, zb, yb, nparam, u,
                               ubar, nsub) != 0)
            return -1;
        for (int tr = 0; tr < ntracer; tr++)
            for (int k = 0; k < L; k++) ybar_out[(size_t)tr * n + s0 + k] += yb[tr * L + k];
    }
    return 0;
}

/* Gradient of the year map: given ybar1 (cotangent of y1 = phi(y0; u)), ybar0 = phi_y^T ybar1
 * and ubar = phi_u^T ybar1.  Stores every state of the year (plain and memory hungry). */
int oracle_year_adjoint(const oracle_problem *P, int model, int ntracer, const double *y0,
                        const double *u, int nparam, int nsub, const double *ybar1, double *ybar0,
                        double *ubar)
{
    size_t len = (size_t)ntracer * P->n;
    double *states = (double *)malloc(sizeof(double) * len * (size_t)P->nstep);
    double *work = (double *)malloc(sizeof(double) * len);
    double *ya = (double *)malloc(sizeof(double) * len), *yb = (double *)malloc(sizeof(double) * len);
    int rc = (states && work && ya && yb) ? 0 : -2;
    if (rc == 0) {
        memcpy(states, y0, sizeof(double) * len);
        for (int j = 0; j + 1 < P->nstep && rc == 0; j++)
            rc = oracle_step(P, model, ntracer, j, states + len * j, states + len * (j + 1), u, nparam, nsub, work);
        for (int k = 0; k < nparam; k++) ubar[k] = 0.0;
        memcpy(ya, ybar1, sizeof(double) * len);
        for (int j = P->nstep - 1; j >= 0 && rc == 0; j--) {
            rc = oracle_step_adjoint(P, model, ntracer, j, states + len * j, ya, yb, u, nparam, ubar, nsub, work);
            double *tmp = ya; ya = yb; yb = tmp;
        }
        memcpy(ybar0, ya, sizeof(double) * len);
    }
    free(states); free(work); free(ya); free(yb);
    return rc;
}
