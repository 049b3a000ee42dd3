// tmm_kernels.cuh -- device code of the TMM step (Metos3D, arXiv:1410.0204, Section 3):
//     y_{j+1} = A_imp(t_j) ( A_exp(t_j) y_j + q_j(y_j, u) ),
// fused into one pass per tile of water columns.  FP64 throughout.
//
// GB300 facts that shape this code: the FP64 pipe retires about one warp-wide DFMA every
// 16 clocks per SM (measured 1.2 TFLOP/s for the whole GPU, 64x below FP32), and a warp
// instruction costs the same whether 1 or 32 lanes are active.  So the year map is bound
// by FP64 instruction issue, not by HBM: every FP64 instruction here is laid out so that
// all 32 lanes do useful work, and transcendentals are hoisted out of the step into
// per-init (insolation) and per-call (light attenuation, Martin profile) tables.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace m3d {

constexpr int kThreads = 256;        // threads per tile CTA
constexpr int kModelNone = 0;
constexpr int kModelNdop = 2;
constexpr double kSigmaPar = 0.4;    // photosynthetically available fraction of I_SWR
constexpr int kEuphotic = 2;         // euphotic layers (Section 7: two)

// One tile: a contiguous range of whole water columns, processed by one CTA.
struct Tile {
    int cell0, ncell;                // cells [cell0, cell0 + ncell)
    int sp0, sp1;                    // explicit-matrix warp slices [sp0, sp1)
    int bk0, bk1;                    // implicit-block warp slices [bk0, bk1)
    int pad0, pad1;
};

// Everything one step reads, as device pointers owned by the context.
struct StepParams {
    int n, nstep, nmonth, nsub, nulat, zmax;
    const Tile *tiles;
    // explicit matrices in warp-slice layout: slice s covers 32 rows (one per lane) and
    // sp_len[s] slots; element (slot q, lane l) of slice s sits at (sp_off[s] + q) * 32 + l.
    const int *sp_len, *sp_off, *sp_row;   // sp_row[s*32+l]: tile-local row or -1
    const int *sp_col;                     // [slots*32] global column index (padding: a valid cell)
    const double *sp_a, *sp_d;             // [nmonth][slots*32]: A_m and A_{m+1} - A_m
    long long sp_mstride;
    // implicit blocks in warp-slice layout: lane l of slice s owns tile-local row bk_row,
    // whose column starts at tile-local cell bk_cb and has bk_L layers; element (c, l) at
    // (bk_off[s] + c) * 32 + l holds B[row][c] (0 beyond bk_L).
    const int *bk_len, *bk_off, *bk_row, *bk_cb, *bk_L;
    const double *bk_b, *bk_d;             // [nmonth][...]: B_m and B_{m+1} - B_m
    long long bk_mstride;
    // biogeochemistry
    const int *cell_kl;                    // layer k | (column layers L << 8)
    const int *cell_ulat;                  // index of the cell's latitude in the insolation table
    const double *h;                       // [n] layer thickness
    const double *atten;                   // [n] sigma_PAR exp(-k_w d) (euphotic cells; per call)
    const double *mfrac;                   // [n] Martin deposition profile (aphotic cells; per call)
    const double *I0tab;                   // [nstep][nulat] daily-mean I_SWR at t_j
    const double *u;                       // [nparam] model parameters
};

// Month weights (Section 3): month m is centred at t = (m + 1/2)/nmonth; t_j = j/nstep.
// s = nmonth t_j - 1/2 = num/den with num = 2 nmonth j - nstep, den = 2 nstep;
// m0 = floor(s) mod nmonth, w = s - floor(s) in [0, 1); the operator is M_m0 + w (M_m1 - M_m0).
__device__ __forceinline__ void month_weights(int j, int nstep, int nmonth, int &m0, double &w)
{
    long long num = 2LL * nmonth * j - nstep;
    long long den = 2LL * nstep;
    long long k = num / den;
    if (num % den != 0 && num < 0) k -= 1;
    long long r = num - k * den;
    m0 = (int)(((k % nmonth) + nmonth) % nmonth);
    w = (double)r / (double)den;
}

// Daily-mean top-of-atmosphere insolation of a circular orbit, the I_SWR forcing of the
// PO4-DOP model (Section 2.2.1 cites Paltridge & Platt without the formula):
// Q = S0/pi (h0 sin(phi) sin(delta) + cos(phi) cos(delta) sin(h0)),
// h0 = arccos(clamp(-tan(phi) tan(delta))), delta = -23.44 deg cos(2 pi (t + 10/360)).
__device__ __forceinline__ double insolation(double lat_deg, double t)
{
    const double pi = 3.14159265358979323846;
    double phi = lat_deg * (pi / 180.0);
    double delta = -23.44 * (pi / 180.0) * cos(2.0 * pi * (t + 10.0 / 360.0));
    double x = -tan(phi) * tan(delta);
    x = fmin(1.0, fmax(-1.0, x));
    double h0 = acos(x);
    return 1361.0 / pi * (h0 * sin(phi) * sin(delta) + cos(phi) * cos(delta) * sin(h0));
}

// PO4-DOP euphotic cell over nsub internal steps (Section 2.2.1), light I fixed:
//   f = alpha N/(N+K_N) I/(I+K_I),  dN = -f + lambda DOP,  dDOP = sigma f - lambda DOP.
// Returns the increments and the production summed over the internal steps.
__device__ __forceinline__ void ndop_euphotic(double N, double D, double I, double alpha,
                                              double sigma, double lambda, double KN, double KI,
                                              double ds, int nsub, double &dN, double &dD,
                                              double &fsum)
{
    double aLF = alpha * (I / (I + KI));
    double N0 = N, D0 = D;
    fsum = 0.0;
    for (int s = 0; s < nsub; s++) {
        double f = aLF * (N / (N + KN));
        double lD = lambda * D;
        N = N + ds * (lD - f);
        D = D + ds * (sigma * f - lD);
        fsum += f;
    }
    dN = N - N0;
    dD = D - D0;
}

// Aphotic PO4-DOP cell: DOP remineralises at lambda; the sinking flux deposits
// Esum * mfrac per unit of production-time (Esum = sum over internal steps of the export).
__device__ __forceinline__ void ndop_aphotic(double D, double Esum, double mfrac, double lambda,
                                             double ds, int nsub, double &dN, double &dD)
{
    double D0 = D, Dsum = 0.0;
    for (int s = 0; s < nsub; s++) {
        Dsum += D;
        D = D + ds * (-(lambda * D));
    }
    dN = ds * (lambda * Dsum + mfrac * Esum);
    dD = D - D0;
}

// Martin profile factor of aphotic layer k of a column: the fraction of the export E
// deposited per metre, ((z_top/z_eu)^-b - (z_bot/z_eu)^-b) / h with the flux through the
// column's bottom interface kept in the bottom layer.
__device__ __forceinline__ double martin_fraction(const double *hcol, int k, int L, double b)
{
    double zeu = hcol[0] + hcol[1];
    double ztop = zeu;
    for (int i = kEuphotic; i < k; i++) ztop += hcol[i];
    double zbot = ztop + hcol[k];
    double ftop = pow(ztop / zeu, -b);
    double fbot = (k == L - 1) ? 0.0 : pow(zbot / zeu, -b);
    return (ftop - fbot) / hcol[k];
}

// A whole shallow column (L <= number of euphotic layers) on one thread, with the export
// kept in its bottom layer inside every internal step.
__device__ __forceinline__ void ndop_shallow_column(int L, const double *hcol, const double *N0,
                                                    const double *D0, const double *I, double alpha,
                                                    double sigma, double lambda, double KN,
                                                    double KI, double ds, int nsub, double *dN,
                                                    double *dD)
{
    double N[kEuphotic], D[kEuphotic];
    for (int k = 0; k < L; k++) { N[k] = N0[k]; D[k] = D0[k]; }
    for (int s = 0; s < nsub; s++) {
        double E = 0.0, f[kEuphotic];
        for (int k = 0; k < L; k++) {
            f[k] = alpha * (N[k] / (N[k] + KN)) * (I[k] / (I[k] + KI));
            E += (1.0 - sigma) * f[k] * hcol[k];
        }
        for (int k = 0; k < L; k++) {
            double qN = -f[k] + lambda * D[k];
            if (k == L - 1) qN += E / hcol[k];
            double qD = sigma * f[k] - lambda * D[k];
            N[k] = N[k] + ds * qN;
            D[k] = D[k] + ds * qD;
        }
    }
    for (int k = 0; k < L; k++) { dN[k] = N[k] - N0[k]; dD[k] = D[k] - D0[k]; }
}

template <bool COHERENT>
__device__ __forceinline__ double load_state(const double *p)
{
    // Inside one persistent launch other CTAs write the state: read it from L2.
    if (COHERENT) return __ldcg(p);
    return __ldg(p);
}

// One TMM step on one tile.  smem: (NTR + 1) * zmax doubles.
template <int NTR, int MODEL, bool COHERENT>
__device__ __forceinline__ void step_tile(const StepParams &P, int tile, int j,
                                          const double *__restrict__ y, double *__restrict__ yn,
                                          double *smem)
{
    const Tile T = P.tiles[tile];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int n = P.n;
    const int zmax = P.zmax;
    double *z = smem;                 // [NTR][zmax] A_exp y + dq, tile-local cells
    double *ek = smem + NTR * zmax;   // [zmax] export contributions of euphotic cells

    int m0;
    double w;
    month_weights(j, P.nstep, P.nmonth, m0, w);

    // ---- explicit part: z = (A_m0 + w (A_m1 - A_m0)) y, all tracers per matrix read
    {
        const double *__restrict__ a0 = P.sp_a + (long long)m0 * P.sp_mstride;
        const double *__restrict__ d0 = P.sp_d + (long long)m0 * P.sp_mstride;
        for (int s = T.sp0 + warp; s < T.sp1; s += nwarps) {
            const int len = __ldg(P.sp_len + s);
            const int base = __ldg(P.sp_off + s) * 32 + lane;
            const int row = __ldg(P.sp_row + s * 32 + lane);
            double acc[NTR];
#pragma unroll
            for (int t = 0; t < NTR; t++) acc[t] = 0.0;
#pragma unroll 4
            for (int q = 0; q < len; q++) {
                const int idx = base + q * 32;
                const int col = __ldg(P.sp_col + idx);
                const double a = fma(w, __ldg(d0 + idx), __ldg(a0 + idx));
#pragma unroll
                for (int t = 0; t < NTR; t++)
                    acc[t] = fma(a, load_state<COHERENT>(y + (size_t)t * n + col), acc[t]);
            }
            if (row >= 0) {
#pragma unroll
                for (int t = 0; t < NTR; t++) z[t * zmax + row] = acc[t];
            }
        }
    }
    __syncthreads();

    // ---- source-minus-sink term q on y_j (Section 2.2.1), added as its increment
    if (MODEL == kModelNdop) {
        const double alpha = __ldg(P.u + 1) * 360.0, sigma = __ldg(P.u + 2);
        const double lambda = __ldg(P.u + 3), KN = __ldg(P.u + 4), KI = __ldg(P.u + 5);
        const int nsub = P.nsub;
        const double ds = (1.0 / P.nstep) / nsub;
        const double *I0row = P.I0tab + (size_t)j * P.nulat;
        for (int i = threadIdx.x; i < T.ncell; i += blockDim.x) {
            const int cell = T.cell0 + i;
            const int kl = __ldg(P.cell_kl + cell);
            const int k = kl & 0xff, L = kl >> 8;
            if (L <= kEuphotic) {
                if (k == 0) {
                    double N0[kEuphotic], D0[kEuphotic], I[kEuphotic], dN[kEuphotic], dD[kEuphotic];
                    const double I0 = __ldg(I0row + __ldg(P.cell_ulat + cell));
                    for (int kk = 0; kk < L; kk++) {
                        N0[kk] = load_state<COHERENT>(y + cell + kk);
                        D0[kk] = load_state<COHERENT>(y + n + cell + kk);
                        I[kk] = I0 * __ldg(P.atten + cell + kk);
                    }
                    ndop_shallow_column(L, P.h + cell, N0, D0, I, alpha, sigma, lambda, KN, KI,
                                        ds, nsub, dN, dD);
                    for (int kk = 0; kk < L; kk++) {
                        z[i + kk] += dN[kk];
                        z[zmax + i + kk] += dD[kk];
                    }
                }
            } else if (k < kEuphotic) {
                const double I = __ldg(I0row + __ldg(P.cell_ulat + cell)) * __ldg(P.atten + cell);
                double dN, dD, fsum;
                ndop_euphotic(load_state<COHERENT>(y + cell), load_state<COHERENT>(y + n + cell), I,
                              alpha, sigma, lambda, KN, KI, ds, nsub, dN, dD, fsum);
                z[i] += dN;
                z[zmax + i] += dD;
                ek[i] = (1.0 - sigma) * fsum * __ldg(P.h + cell);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < T.ncell; i += blockDim.x) {
            const int cell = T.cell0 + i;
            const int kl = __ldg(P.cell_kl + cell);
            const int k = kl & 0xff, L = kl >> 8;
            if (L > kEuphotic && k >= kEuphotic) {
                const double Esum = ek[i - k] + ek[i - k + 1];
                double dN, dD;
                ndop_aphotic(load_state<COHERENT>(y + n + cell), Esum, __ldg(P.mfrac + cell), lambda,
                             ds, nsub, dN, dD);
                z[i] += dN;
                z[zmax + i] += dD;
            }
        }
        __syncthreads();
    }

    // ---- implicit part: y_{j+1} = (B_m0 + w (B_m1 - B_m0)) z, column by column
    {
        const double *__restrict__ b0 = P.bk_b + (long long)m0 * P.bk_mstride;
        const double *__restrict__ bd = P.bk_d + (long long)m0 * P.bk_mstride;
        for (int s = T.bk0 + warp; s < T.bk1; s += nwarps) {
            const int len = __ldg(P.bk_len + s);
            const int base = __ldg(P.bk_off + s) * 32 + lane;
            const int row = __ldg(P.bk_row + s * 32 + lane);
            const int cb = __ldg(P.bk_cb + s * 32 + lane);
            const int Lc = __ldg(P.bk_L + s * 32 + lane);
            double acc[NTR];
#pragma unroll
            for (int t = 0; t < NTR; t++) acc[t] = 0.0;
#pragma unroll 4
            for (int c = 0; c < len; c++) {
                const int idx = base + c * 32;
                const double b = fma(w, __ldg(bd + idx), __ldg(b0 + idx));
                const int zi = cb + (c < Lc ? c : 0);
#pragma unroll
                for (int t = 0; t < NTR; t++) acc[t] = fma(b, z[t * zmax + zi], acc[t]);
            }
            if (row >= 0) {
#pragma unroll
                for (int t = 0; t < NTR; t++) yn[(size_t)t * n + T.cell0 + row] = acc[t];
            }
        }
    }
}

}  // namespace m3d
