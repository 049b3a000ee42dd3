// ensemble.cu -- batched ensembles: many members (model + parameters) advanced together through
// the TMM steps of Metos3D (arXiv:1410.0204, Section 3), one kernel launch per step and one
// CUDA graph per model year (Section 4).
//
// Layout.  The members' tracers are packed into groups of 32 lanes (no member split between
// groups; first fit, members with more tracers first) and the state is stored cell-major,
// X[cell][group * 32 + lane], so that a warp reading one cell of one group reads 256
// contiguous bytes.  Lanes that hold no tracer stay zero.
//
// Step kernel.  A CTA takes a block of consecutive water columns.  It interpolates the
// explicit matrix rows of its cells once per step into shared memory,
// A(t_j) = A_m0 + w (A_m1 - A_m0), and stages the Thomas factors of both months of its cells;
// every tracer of every member then reuses them.  Its warps take (column, group) items from a
// shared counter; for its item a warp, one lane per tracer,
//   1. reads y_j of the column and forms z = A_exp(t_j) y_j row by row (one FMA per entry);
//   2. evaluates the members' source terms q(y_j) with the lanes re-dealt to (member, layer)
//      pairs -- the models' per-cell work is then done once per member, not once per tracer --
//      and adds dt q (or the nsub-step increment) to z;
//   3. applies the interpolated implicit operator, (1 - w) T0^-1 z + w T1^-1 z with T_h the
//      tridiagonal matrix whose inverse is month h's block (Thomas solves), and writes y_{j+1}.
// Nothing waits on another CTA, so a step is one ordinary launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "metos3d.h"
#include "tmm_kernels.cuh"
#include "context.h"

namespace {

constexpr int kLanes = 32;
constexpr int kParSlots = 16;             // derived model scalars per member
constexpr int kMaxWarps = 16;
constexpr unsigned kFull = 0xffffffffu;
constexpr double kSigmaPar = 0.4;         // photosynthetically available fraction of I_SWR

// Slots of the derived member scalars (host-computed from the user's parameters).
//   every model: [0] k_w, [1] b (Martin models)
//   N:    [2] alpha', [3] K_N, [4] K_I
//   NDOP: [2] alpha', [3] K_N, [4] K_I, [5] sigma, [6] lambda, [7] 1 - sigma
//   PHY:  [2] mu_1', [3] K_1, [4] K_I, [5] lambda'_2, [6] sigma_2, [7] lambda_3', [8] kappa_3',
//         [9] lambda'_3', [10] sigma_3, [11] 1 - sigma_3, [12] 1 - sigma_2
//   NPZD: [2] mu_P', [3] K_N, [4] K_I, [5] mu_Z', [6] K_P, [7] epsilon, [8] lambda_P', [9] kappa_Z',
//         [10] lambda_Z', [11] lambda_D', [12] lambda_DOP', [13] w_D', [14] 1 - epsilon
// (primes: per year, the per-day rates times 360).

struct EnsParams {
    int n, ncol, nstep, nmonth, nsub, wp, ngroup, nulat, zmax;
    int cpb, nnz_blk_max, cells_blk_max;
    double ds;                            // internal model step (1 / nstep) / nsub
    const int *m0tab;                     // [nstep]
    const double *wtab;                   // [nstep]
    const int *rowptr, *colidx;           // explicit pattern (CSR)
    const double *ea, *ed;                // [nmonth][nnz]: A_m and A_{m+1} - A_m
    long long e_mstride;
    const double *tri;                    // [nmonth][3][n] Thomas factors (-l_k, 1/d_k, -e_k/d_{k+1})
    long long tri_mstride;
    const int *col_start, *col_ulat;
    const double *h;
    const double *I0tab;                  // [nstep][nulat]
    const int *grp_seg_off;               // [ngroup + 1] segments of each group
    const int4 *segs;                     // (model, first member slot, end member slot, 0)
    const int *mem_lane0, *mem_pidx;      // per member slot: first lane in its group, member index
    const double *mpar;                   // [nmember][kParSlots]
    const double *atten;                  // [nmember][ncol][2] sigma_PAR exp(-k_w d) of the euphotic cells
    const double *mfrac;                  // [nmember][n] Martin deposition profile (Martin models)
};

// Shared-memory layout of the step kernel (doubles first, then ints).
__host__ __device__ inline size_t ens_warp_doubles(int zmax, bool sub1)
{
    return (size_t)(sub1 ? 2 : 4) * zmax * kLanes + kLanes;
}
__host__ __device__ inline size_t ens_smem_bytes(int nnz_blk_max, int cells_blk_max, int zmax, int nwarps, bool sub1)
{
    return sizeof(double) * ((size_t)nnz_blk_max + 6 * (size_t)cells_blk_max + nwarps * ens_warp_doubles(zmax, sub1)) +
           sizeof(int) * ((size_t)nnz_blk_max + 4);
}

// A member's tracer t at layer k of the column's staging array st: the value, or for a
// member that carries its tangent (T = Dual) the value and its perturbation, which sits
// ntr lanes further on.
template <class T> struct EnsLane;
template <> struct EnsLane<double> {
    __device__ __forceinline__ static double get(const double *st, int k, int l0, int t, int)
    {
        return st[k * kLanes + l0 + t];
    }
    // the increment: z += ds q (one internal step) or q into the substep buffer
    template <bool SUB1>
    __device__ __forceinline__ static void emit(double *zs, double *qs, double ds, int k, int l0, int t, int, double q)
    {
        if (SUB1) zs[k * kLanes + l0 + t] = fma(ds, q, zs[k * kLanes + l0 + t]);
        else qs[k * kLanes + l0 + t] = q;
    }
    __device__ __forceinline__ static double madd(double a, double b, double c) { return fma(a, b, c); }
    __device__ __forceinline__ static double partner_sum(double e) { return e + __shfl_xor_sync(kFull, e, 1); }
    __device__ __forceinline__ static void put_export(double *Es, int ml, double v) { Es[ml] = v; }
    __device__ __forceinline__ static double get_export(const double *Es, int ml) { return Es[ml]; }
};
template <> struct EnsLane<m3d::Dual> {
    __device__ __forceinline__ static m3d::Dual get(const double *st, int k, int l0, int t, int ntr)
    {
        return {st[k * kLanes + l0 + t], st[k * kLanes + l0 + ntr + t]};
    }
    template <bool SUB1>
    __device__ __forceinline__ static void emit(double *zs, double *qs, double ds, int k, int l0, int t, int ntr,
                                                m3d::Dual q)
    {
        EnsLane<double>::emit<SUB1>(zs, qs, ds, k, l0, t, 0, q.v);
        EnsLane<double>::emit<SUB1>(zs, qs, ds, k, l0 + ntr, t, 0, q.d);
    }
    __device__ __forceinline__ static m3d::Dual madd(m3d::Dual a, double b, m3d::Dual c) { return a * b + c; }
    __device__ __forceinline__ static m3d::Dual partner_sum(m3d::Dual e)
    {
        return {e.v + __shfl_xor_sync(kFull, e.v, 1), e.d + __shfl_xor_sync(kFull, e.d, 1)};
    }
    __device__ __forceinline__ static void put_export(double *Es, int ml, m3d::Dual v)
    {
        Es[2 * ml] = v.v;
        Es[2 * ml + 1] = v.d;
    }
    __device__ __forceinline__ static m3d::Dual get_export(const double *Es, int ml) { return {Es[2 * ml], Es[2 * ml + 1]}; }
};

// The source terms of one segment (members of one model in one lane group) on one column,
// the warp's lanes dealt to (member, layer) pairs.  T = double: the models; T = Dual: the
// models and their tangents, for members that carry a perturbation in the ntr lanes after
// their state.
template <class T, bool SUB1>
__device__ __forceinline__ void ens_segment_q(const EnsParams &E, const int4 &S, int c, int s0, int L, double I0,
                                              int lane, const double *st, double *zs, double *qs, double *Es)
{
    typedef EnsLane<T> A;
    const int model = S.x, nm = S.z - S.y;
    const int neu = L < 2 ? L : 2, na = L - neu;
    const double ds = E.ds;
    if (model == M3D_MODEL_NPZD) {
        const int ntr = 5;
        for (int base = 0; base < nm * L; base += kLanes) {
            const int p = base + lane;
            if (p >= nm * L) continue;
            const int ml = p / L, k = p - ml * L, mi = S.y + ml;
            const int l0 = E.mem_lane0[mi], pid = E.mem_pidx[mi];
            const double *mp = E.mpar + (size_t)pid * kParSlots;
            const T N = A::get(st, k, l0, 0, ntr), P = A::get(st, k, l0, 1, ntr);
            const T Z = A::get(st, k, l0, 2, ntr), D = A::get(st, k, l0, 3, ntr);
            const T DOP = A::get(st, k, l0, 4, ntr);
            // one division for both rates: U = mu_P P N/(N+K_N) I/(I+K_I) (I = 0 below
            // the euphotic zone) and G = mu_Z Z P/(K_P+P)
            const double I = k < neu ? I0 * E.atten[((size_t)pid * E.ncol + c) * 2 + k] : 0.0;
            const T dN = N + mp[3];
            const double dI = I + mp[4];
            const T dP = mp[6] + P;
            const T dNI = dN * dI;
            T U, G;
            if constexpr (std::is_same<T, double>::value) {
                const T r = 1.0 / (dNI * dP);
                U = mp[2] * P * N * I * dP * r;
                G = mp[5] * Z * P * dNI * r;
            } else {
                // on dual numbers a shared division would cancel (the derivative of dP / (dNI dP)
                // takes two large terms of opposite sign): one division per rate
                U = mp[2] * P * N * I / dNI;
                G = mp[5] * Z * P / dP;
            }
            const T mP = mp[8] * P, mZ = mp[9] * Z * Z, eZ = mp[10] * Z;
            const T rD = mp[11] * D, rO = mp[12] * DOP;
            const T zero{};
            const T Sin = k > 0 ? mp[13] * A::get(st, k - 1, l0, 3, ntr) : zero;
            const T Sout = k + 1 < L ? mp[13] * D : zero;
            const double hk = E.h[s0 + k];
            A::template emit<SUB1>(zs, qs, ds, k, l0, 0, ntr, -U + rO);
            A::template emit<SUB1>(zs, qs, ds, k, l0, 1, ntr, U - G - mP);
            A::template emit<SUB1>(zs, qs, ds, k, l0, 2, ntr, mp[7] * G - mZ - eZ);
            A::template emit<SUB1>(zs, qs, ds, k, l0, 3, ntr, mP + mZ - rD + (Sin - Sout) / hk);
            A::template emit<SUB1>(zs, qs, ds, k, l0, 4, ntr, mp[14] * G + eZ + rD - rO);
        }
        return;
    }
    // Martin models (N, NDOP, PHY): euphotic pairs, export E reduced over the member's
    // euphotic layers (adjacent lanes), then the aphotic pairs
    const int ntr = model == M3D_MODEL_N ? 1 : model == M3D_MODEL_NDOP ? 2 : 3;
    for (int base = 0; base < nm * neu; base += kLanes) {
        const int p = base + lane;
        const bool act = p < nm * neu;
        const int ml = act ? p / neu : 0, k = act ? p - ml * neu : 0, mi = S.y + ml;
        T e{}, q0{}, q1{}, q2{};
        int l0 = 0, pid = 0;
        if (act) {
            l0 = E.mem_lane0[mi];
            pid = E.mem_pidx[mi];
            const double *mp = E.mpar + (size_t)pid * kParSlots;
            const double I = I0 * E.atten[((size_t)pid * E.ncol + c) * 2 + k];
            const double hk = E.h[s0 + k];
            const T N = A::get(st, k, l0, 0, ntr);
            // both half-saturation factors with one division
            const T lim = (N * I) / ((N + mp[3]) * (I + mp[4]));
            if (model == M3D_MODEL_N) {
                const T f = mp[2] * lim;
                q0 = -f;
                e = f * hk;
            } else if (model == M3D_MODEL_NDOP) {
                const T DOP = A::get(st, k, l0, 1, ntr);
                const T f = mp[2] * lim;
                q0 = -f + mp[6] * DOP;
                q1 = mp[5] * f - mp[6] * DOP;
                e = mp[7] * f * hk;
            } else {                                   // PHY
                const T DOP = A::get(st, k, l0, 1, ntr), PHY = A::get(st, k, l0, 2, ntr);
                const T f1 = mp[2] * PHY * lim;
                const T f3 = mp[10] * f1;
                const T loss = mp[7] * PHY + mp[8] * PHY * PHY;
                q0 = -f1 + mp[5] * DOP;
                q1 = mp[6] * f3 + loss - mp[5] * DOP + mp[9] * PHY;
                q2 = mp[11] * f1 - loss - mp[9] * PHY;
                e = mp[12] * f3 * hk;
            }
        }
        const T Eg = neu == 2 ? A::partner_sum(e) : e;
        if (act) {
            if (L <= 2 && k == L - 1) q0 = A::madd(Eg, E.mfrac[(size_t)pid * E.n + s0 + k], q0);
            if (k == 0) A::put_export(Es, ml, Eg);
            A::template emit<SUB1>(zs, qs, ds, k, l0, 0, ntr, q0);
            if (model != M3D_MODEL_N) A::template emit<SUB1>(zs, qs, ds, k, l0, 1, ntr, q1);
            if (model == M3D_MODEL_PHY) A::template emit<SUB1>(zs, qs, ds, k, l0, 2, ntr, q2);
        }
    }
    __syncwarp();
    for (int base = 0; base < nm * na; base += kLanes) {
        const int p = base + lane;
        if (p >= nm * na) continue;
        const int ml = p / na, k = neu + (p - ml * na), mi = S.y + ml;
        const int l0 = E.mem_lane0[mi], pid = E.mem_pidx[mi];
        const double *mp = E.mpar + (size_t)pid * kParSlots;
        const T dep = A::get_export(Es, ml) * E.mfrac[(size_t)pid * E.n + s0 + k];
        if (model == M3D_MODEL_N) {
            A::template emit<SUB1>(zs, qs, ds, k, l0, 0, ntr, dep);
        } else if (model == M3D_MODEL_NDOP) {
            const T DOP = A::get(st, k, l0, 1, ntr);
            A::template emit<SUB1>(zs, qs, ds, k, l0, 0, ntr, dep + mp[6] * DOP);
            A::template emit<SUB1>(zs, qs, ds, k, l0, 1, ntr, -(mp[6] * DOP));
        } else {
            const T DOP = A::get(st, k, l0, 1, ntr), PHY = A::get(st, k, l0, 2, ntr);
            A::template emit<SUB1>(zs, qs, ds, k, l0, 0, ntr, dep + mp[5] * DOP);
            A::template emit<SUB1>(zs, qs, ds, k, l0, 1, ntr, -(mp[5] * DOP) + mp[9] * PHY);
            A::template emit<SUB1>(zs, qs, ds, k, l0, 2, ntr, -(mp[9] * PHY));
        }
    }
    __syncwarp();
}

template <bool SUB1>
__global__ void __launch_bounds__(kMaxWarps * kLanes) k_ens_step(EnsParams E, int j, const double *__restrict__ X,
                                                                 double *__restrict__ Xn)
{
    extern __shared__ double smem[];
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = blockIdx.x * E.cpb, c1 = min(c0 + E.cpb, E.ncol);
    const int cell0 = E.col_start[c0], cell1 = E.col_start[c1];
    const int p0 = E.rowptr[cell0], p1 = E.rowptr[cell1];
    const int cbm = E.cells_blk_max, zm = E.zmax;

    double *sval = smem;
    double *stri = sval + E.nnz_blk_max;
    double *wb = stri + 6 * cbm + (size_t)warp * ens_warp_doubles(zm, SUB1);
    double *ys = wb, *zs = ys + zm * kLanes;
    double *yw = SUB1 ? ys : zs + zm * kLanes;
    double *qs = SUB1 ? zs : yw + zm * kLanes;
    double *Es = wb + (SUB1 ? 2 : 4) * zm * kLanes;
    int *scol = (int *)(stri + 6 * cbm + (size_t)nw * ens_warp_doubles(zm, SUB1));
    int *counter = scol + E.nnz_blk_max;

    const int m0 = E.m0tab[j], m1 = (m0 + 1) % E.nmonth;
    const double w = E.wtab[j];
    {
        const double *a0 = E.ea + (size_t)m0 * E.e_mstride, *d0 = E.ed + (size_t)m0 * E.e_mstride;
        for (int p = threadIdx.x; p < p1 - p0; p += blockDim.x) {
            sval[p] = fma(w, d0[p0 + p], a0[p0 + p]);
            scol[p] = E.colidx[p0 + p];
        }
        // Thomas factors of both months; the blend (1 - w) T0^-1 z + w T1^-1 z is folded into the
        // reciprocal pivots, which scale the two back substitutions' unknowns u_k = d_k y_k
        const double *t0 = E.tri + (size_t)m0 * E.tri_mstride, *t1 = E.tri + (size_t)m1 * E.tri_mstride;
        for (int i = threadIdx.x; i < cell1 - cell0; i += blockDim.x)
            for (int f = 0; f < 3; f++) {
                const double a = t0[(size_t)f * E.n + cell0 + i], b = t1[(size_t)f * E.n + cell0 + i];
                stri[f * cbm + i] = f == 1 ? (1.0 - w) * a : a;
                stri[(3 + f) * cbm + i] = f == 1 ? w * b : b;
            }
        if (threadIdx.x == 0) *counter = 0;
    }
    __syncthreads();

    const int nitems = (c1 - c0) * E.ngroup;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(counter, 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= nitems) break;
        const int c = c0 + item / E.ngroup, g = item - (item / E.ngroup) * E.ngroup;
        const int s0 = E.col_start[c], L = E.col_start[c + 1] - s0, sl = s0 - cell0;
        const size_t gl = (size_t)g * kLanes + lane;

        // 1. y_j of the column and z = A_exp(t_j) y_j
        for (int k = 0; k < L; k++) ys[k * kLanes + lane] = X[(size_t)(s0 + k) * E.wp + gl];
        for (int k = 0; k < L; k++) {
            const int pb = E.rowptr[s0 + k] - p0, pe = E.rowptr[s0 + k + 1] - p0;
            double z = 0.0;
            int p = pb;
            for (; p + 1 < pe; p += 2) {
                const double xa = X[(size_t)scol[p] * E.wp + gl], xb = X[(size_t)scol[p + 1] * E.wp + gl];
                z = fma(sval[p], xa, z);
                z = fma(sval[p + 1], xb, z);
            }
            if (p < pe) z = fma(sval[p], X[(size_t)scol[p] * E.wp + gl], z);
            zs[k * kLanes + lane] = z;
        }
        if (!SUB1) {
            for (int k = 0; k < L; k++) {
                yw[k * kLanes + lane] = ys[k * kLanes + lane];
                qs[k * kLanes + lane] = 0.0;
            }
        }
        __syncwarp();

        // 2. source terms, lanes over (member, layer) pairs
        const double I0 = E.I0tab[(size_t)j * E.nulat + E.col_ulat[c]];
        const int sg0 = E.grp_seg_off[g], sg1 = E.grp_seg_off[g + 1];
        for (int sub = 0; sub < (SUB1 ? 1 : E.nsub); sub++) {
            const double *st = SUB1 ? ys : yw;
            for (int sg = sg0; sg < sg1; sg++) {
                const int4 S = E.segs[sg];
                if (S.w) ens_segment_q<m3d::Dual, SUB1>(E, S, c, s0, L, I0, lane, st, zs, qs, Es);
                else ens_segment_q<double, SUB1>(E, S, c, s0, L, I0, lane, st, zs, qs, Es);
            }
            if (!SUB1) {
                __syncwarp();
                for (int k = 0; k < L; k++) yw[k * kLanes + lane] = fma(E.ds, qs[k * kLanes + lane], yw[k * kLanes + lane]);
                __syncwarp();
            }
        }
        if (!SUB1) {
            for (int k = 0; k < L; k++) zs[k * kLanes + lane] += yw[k * kLanes + lane] - ys[k * kLanes + lane];
        }
        __syncwarp();

        // 3. implicit part: Thomas solves of both months, then z0 + w (z1 - z0)
        {
            const double *nl0 = stri + sl, *rd0 = stri + cbm + sl, *ne0 = stri + 2 * cbm + sl;
            const double *nl1 = stri + 3 * cbm + sl, *rd1 = stri + 4 * cbm + sl, *ne1 = stri + 5 * cbm + sl;
            double g0 = 0.0, g1 = 0.0;
            for (int k = 0; k < L; k++) {
                const double z = zs[k * kLanes + lane];
                g0 = fma(nl0[k], g0, z);
                g1 = fma(nl1[k], g1, z);
                ys[k * kLanes + lane] = g0;
                zs[k * kLanes + lane] = g1;
            }
            // back substitution in u_k = d_k y_k (third factor -e_k/d_{k+1}); the staged pivots
            // carry the blend weights, (1 - w)/d_k and w/d_k
            double u0 = 0.0, u1 = 0.0;
            for (int k = L - 1; k >= 0; k--) {
                u0 = fma(ne0[k], u0, ys[k * kLanes + lane]);
                u1 = fma(ne1[k], u1, zs[k * kLanes + lane]);
                Xn[(size_t)(s0 + k) * E.wp + gl] = fma(rd0[k], u0, rd1[k] * u1);
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------------------------
// Reverse (adjoint) ensemble step, one internal model step (Section 6's exact derivatives, by
// hand).  For y_{j+1} = B_j (A_j y_j + ds q(y_j)) and the cotangent ybar_{j+1}:
//   zbar_j = B_j^T ybar_{j+1}                                   (k_ens_adj_implicit)
//   ybar_j = A_j^T zbar_j + ds (dq/dy)^T zbar_j,  ubar += ds (dq/du)^T zbar_j   (k_ens_adj_explicit)
// A_j^T has the explicit pattern's transpose, which the structurally symmetric pattern shares:
// its values sit in the same CSR slots.  B_j^T = (1 - w) T0^-T + w T1^-T with T_h^T tridiagonal.
struct EnsAdjParams {
    const double *eat, *edt;              // [nmonth][nnz] A_m^T and A_{m+1}^T - A_m^T in the CSR slots
    const double *trit;                   // [nmonth][3][n] Thomas factors of T_m^T (back-substitution form)
    const double *mfrac_b;                // [nmember][n] d mfrac / d b (Martin models)
    double *ub_part;                      // [nblocks][nmember][kParSlots] gradient in the derived slots
    int nmember;
};

// zbar_j = B_j^T ybar on every (column, group) item; ybar, zbar packed [n][wp].
__global__ void __launch_bounds__(kMaxWarps * kLanes) k_ens_adj_implicit(EnsParams E, EnsAdjParams A, int j,
                                                                         const double *__restrict__ Yb,
                                                                         double *__restrict__ Zb)
{
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = blockIdx.x * E.cpb, c1 = min(c0 + E.cpb, E.ncol);
    const int cell0 = E.col_start[c0], cell1 = E.col_start[c1];
    const int cbm = E.cells_blk_max, zm = E.zmax;
    double *stri = smem;
    double *wb = stri + 6 * cbm + (size_t)warp * 2 * zm * kLanes;
    double *ys = wb, *zs = ys + zm * kLanes;
    int *counter = (int *)(stri + 6 * cbm + (size_t)(blockDim.x >> 5) * 2 * zm * kLanes);
    const int m0 = E.m0tab[j], m1 = (m0 + 1) % E.nmonth;
    const double w = E.wtab[j];
    {
        const double *t0 = A.trit + (size_t)m0 * E.tri_mstride, *t1 = A.trit + (size_t)m1 * E.tri_mstride;
        for (int i = threadIdx.x; i < cell1 - cell0; i += blockDim.x)
            for (int f = 0; f < 3; f++) {
                const double a = t0[(size_t)f * E.n + cell0 + i], b = t1[(size_t)f * E.n + cell0 + i];
                stri[f * cbm + i] = f == 1 ? (1.0 - w) * a : a;
                stri[(3 + f) * cbm + i] = f == 1 ? w * b : b;
            }
        if (threadIdx.x == 0) *counter = 0;
    }
    __syncthreads();
    const int nitems = (c1 - c0) * E.ngroup;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(counter, 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= nitems) break;
        const int c = c0 + item / E.ngroup, g = item - (item / E.ngroup) * E.ngroup;
        const int s0 = E.col_start[c], L = E.col_start[c + 1] - s0, sl = s0 - cell0;
        const size_t gl = (size_t)g * kLanes + lane;
        const double *nl0 = stri + sl, *rd0 = stri + cbm + sl, *ne0 = stri + 2 * cbm + sl;
        const double *nl1 = stri + 3 * cbm + sl, *rd1 = stri + 4 * cbm + sl, *ne1 = stri + 5 * cbm + sl;
        double g0 = 0.0, g1 = 0.0;
        for (int k = 0; k < L; k++) {
            const double yb = Yb[(size_t)(s0 + k) * E.wp + gl];
            g0 = fma(nl0[k], g0, yb);
            g1 = fma(nl1[k], g1, yb);
            ys[k * kLanes + lane] = g0;
            zs[k * kLanes + lane] = g1;
        }
        double u0 = 0.0, u1 = 0.0;
        for (int k = L - 1; k >= 0; k--) {
            u0 = fma(ne0[k], u0, ys[k * kLanes + lane]);
            u1 = fma(ne1[k], u1, zs[k * kLanes + lane]);
            Zb[(size_t)(s0 + k) * E.wp + gl] = fma(rd0[k], u0, rd1[k] * u1);
        }
        __syncwarp();
    }
}

// The sums over the lanes of each member of a pass: lanes p = base + lane belong to member
// (p / per) of the pass, contiguous; after the segmented suffix sums the first lane of each
// member's run in this warp holds the run's total.
__device__ __forceinline__ double member_run_sum(double v, int key, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double other = __shfl_down_sync(kFull, v, o);
        const int okey = __shfl_down_sync(kFull, key, o);
        if (lane + o < 32 && okey == key) v += other;
    }
    return v;
}

// Add a pass's per-lane parameter gradients g[0..np) of member `pid` (the member's index in the
// caller's order; key = member within the pass, -1 for idle lanes) into the block's
// accumulators ub[pid][slot].
__device__ __forceinline__ void add_member_gradients(double *ub, const double *gv, int np, int key, int pid, int lane)
{
    const int prev = __shfl_up_sync(kFull, key, 1);
    const bool head = key >= 0 && (lane == 0 || prev != key);
    for (int q = 0; q < np; q++) {
        const double v = member_run_sum(key >= 0 ? gv[q] : 0.0, key, lane);
        if (head && v != 0.0) atomicAdd(ub + (size_t)pid * kParSlots + q, v);
    }
}

// Reverse of one segment's source terms on one column: qb = ds zbar (own column, zbs), the
// state y_j (ys); adds (dq/dy)^T qb into ybs and (dq/du)^T qb into ub[member slot][derived slot],
// slot 0 holding d/dk_w (through the light attenuation) and slot 1 d/db (through the Martin
// profile).
__device__ __forceinline__ void ens_segment_qadj(const EnsParams &E, const EnsAdjParams &A, const int4 &S, int c,
                                                 int s0, int L, double I0, int lane, const double *ys,
                                                 const double *zbs, double *ybs, double *Es, double *Ebs, double *ub)
{
    const int model = S.x, nm = S.z - S.y;
    const int neu = L < 2 ? L : 2, na = L - neu;
    const double ds = E.ds;
    const double *zc = E.h + E.n;
    auto st = [&](int k, int l0, int t) { return ys[k * kLanes + l0 + t]; };
    auto qb = [&](int k, int l0, int t) { return ds * zbs[k * kLanes + l0 + t]; };
    auto addy = [&](int k, int l0, int t, double v) { ybs[k * kLanes + l0 + t] += v; };
    if (model == M3D_MODEL_NPZD) {
        for (int base = 0; base < nm * L; base += kLanes) {
            const int p = base + lane;
            const bool act = p < nm * L;
            const int ml = act ? p / L : -1, k = act ? p - ml * L : 0, mi = S.y + (act ? ml : 0);
            double gv[15];
#pragma unroll
            for (int q = 0; q < 15; q++) gv[q] = 0.0;
            if (act) {
                const int l0 = E.mem_lane0[mi], pid = E.mem_pidx[mi];
                const double *mp = E.mpar + (size_t)pid * kParSlots;
                const double N = st(k, l0, 0), P = st(k, l0, 1), Z = st(k, l0, 2), D = st(k, l0, 3);
                const double DOP = st(k, l0, 4);
                const double bN = qb(k, l0, 0), bP = qb(k, l0, 1), bZ = qb(k, l0, 2), bD = qb(k, l0, 3);
                const double bO = qb(k, l0, 4);
                const double at = k < neu ? E.atten[((size_t)pid * E.ncol + c) * 2 + k] : 0.0;
                const double I = I0 * at;
                const double dN = N + mp[3], dI = I + mp[4], dP = mp[6] + P;
                // U = mu_P P N I / (dN dI), G = mu_Z Z P / dP
                const double PNI = P * N * I / (dN * dI);
                const double U = mp[2] * PNI;
                const double R = P / dP;
                const double G = mp[5] * Z * R;
                const double Ub = -bN + bP;
                const double Gb = -bP + mp[7] * bZ + mp[14] * bO;
                const double mPb = -bP + bD, mZb = -bZ + bD, eZb = -bZ + bO, rDb = -bD + bO, rOb = bN - bO;
                double yN = 0.0, yP = 0.0, yZ = 0.0, yD = 0.0, yO = 0.0;
                if (k < neu) {
                    yN += Ub * mp[2] * P * I * mp[3] / (dN * dN * dI);
                    yP += Ub * mp[2] * N * I / (dN * dI);
                    gv[2] += Ub * PNI;
                    gv[3] += -Ub * U / dN;
                    gv[4] += -Ub * U / dI;
                    // dU/dI = mu_P P N K_I / (dN dI^2), dI/dk_w = -zc I
                    gv[0] += Ub * (mp[2] * P * N * mp[4] / (dN * dI * dI)) * (-zc[s0 + k] * I);
                }
                yZ += Gb * mp[5] * R;
                yP += Gb * mp[5] * Z * mp[6] / (dP * dP);
                gv[5] += Gb * Z * R;
                gv[6] += -Gb * G / dP;
                gv[7] += G * bZ;
                gv[14] += G * bO;
                yP += mp[8] * mPb;
                gv[8] += mPb * P;
                yZ += 2.0 * mp[9] * Z * mZb + mp[10] * eZb;
                gv[9] += mZb * Z * Z;
                gv[10] += eZb * Z;
                yD += mp[11] * rDb;
                gv[11] += rDb * D;
                yO += mp[12] * rOb;
                gv[12] += rOb * DOP;
                if (k + 1 < L) {        // S_k = w_D D_k leaves layer k into layer k + 1
                    const double Sb = -bD / E.h[s0 + k] + qb(k + 1, l0, 3) / E.h[s0 + k + 1];
                    yD += mp[13] * Sb;
                    gv[13] += D * Sb;
                }
                addy(k, l0, 0, yN);
                addy(k, l0, 1, yP);
                addy(k, l0, 2, yZ);
                addy(k, l0, 3, yD);
                addy(k, l0, 4, yO);
            }
            add_member_gradients(ub, gv, 15, ml, E.mem_pidx[mi], lane);
        }
        return;
    }
    // Martin models: (1) the euphotic lanes recompute the export E of each member, (2) the
    // aphotic lanes (and a shallow column's bottom layer) reverse their terms and sum the
    // export's cotangent Ebar per member, (3) the euphotic lanes reverse with Ebar
    for (int base = 0; base < nm * neu; base += kLanes) {
        const int p = base + lane;
        const bool act = p < nm * neu;
        const int ml = act ? p / neu : 0, k = act ? p - ml * neu : 0, mi = S.y + ml;
        double e = 0.0;
        if (act) {
            const int l0 = E.mem_lane0[mi], pid = E.mem_pidx[mi];
            const double *mp = E.mpar + (size_t)pid * kParSlots;
            const double I = I0 * E.atten[((size_t)pid * E.ncol + c) * 2 + k];
            const double N = st(k, l0, 0);
            const double lim = (N * I) / ((N + mp[3]) * (I + mp[4]));
            const double hk = E.h[s0 + k];
            if (model == M3D_MODEL_N) e = mp[2] * lim * hk;
            else if (model == M3D_MODEL_NDOP) e = mp[7] * (mp[2] * lim) * hk;
            else e = mp[12] * (mp[10] * (mp[2] * st(k, l0, 2) * lim)) * hk;
        }
        const double Eg = neu == 2 ? e + __shfl_xor_sync(kFull, e, 1) : e;
        if (act && k == 0) {
            Es[ml] = Eg;
            Ebs[ml] = 0.0;
        }
    }
    __syncwarp();
    // aphotic layers, and the bottom layer of a shallow column (its export stays there)
    const int nap = na > 0 ? na : 1;
    for (int base = 0; base < nm * nap; base += kLanes) {
        const int p = base + lane;
        const bool act = p < nm * nap;
        const int ml = act ? p / nap : -1, mi = S.y + (act ? ml : 0);
        const int k = na > 0 ? neu + (p - (act ? ml : 0) * nap) : L - 1;
        double gv[13];
#pragma unroll
        for (int q = 0; q < 13; q++) gv[q] = 0.0;
        if (act) {
            const int l0 = E.mem_lane0[mi], pid = E.mem_pidx[mi];
            const double *mp = E.mpar + (size_t)pid * kParSlots;
            const double Ev = Es[ml];
            const double mf = E.mfrac[(size_t)pid * E.n + s0 + k];
            const double b0 = qb(k, l0, 0);
            double Ebp = b0 * mf;
            gv[1] += b0 * Ev * A.mfrac_b[(size_t)pid * E.n + s0 + k];
            if (na > 0) {
                if (model == M3D_MODEL_NDOP) {
                    const double b1 = qb(k, l0, 1), DOP = st(k, l0, 1);
                    addy(k, l0, 1, mp[6] * (b0 - b1));
                    gv[6] += (b0 - b1) * DOP;
                } else if (model == M3D_MODEL_PHY) {
                    const double b1 = qb(k, l0, 1), b2 = qb(k, l0, 2);
                    const double DOP = st(k, l0, 1), PHY = st(k, l0, 2);
                    addy(k, l0, 1, mp[5] * (b0 - b1));
                    gv[5] += (b0 - b1) * DOP;
                    addy(k, l0, 2, mp[9] * (b1 - b2));
                    gv[9] += (b1 - b2) * PHY;
                }
            }
            atomicAdd(Ebs + ml, Ebp);
        }
        add_member_gradients(ub, gv, 13, ml, E.mem_pidx[mi], lane);
    }
    __syncwarp();
    for (int base = 0; base < nm * neu; base += kLanes) {
        const int p = base + lane;
        const bool act = p < nm * neu;
        const int ml = act ? p / neu : -1, k = act ? p - ml * neu : 0, mi = S.y + (act ? ml : 0);
        double gv[13];
#pragma unroll
        for (int q = 0; q < 13; q++) gv[q] = 0.0;
        if (act) {
            const int l0 = E.mem_lane0[mi], pid = E.mem_pidx[mi];
            const double *mp = E.mpar + (size_t)pid * kParSlots;
            const double Eb = Ebs[ml];
            const double I = I0 * E.atten[((size_t)pid * E.ncol + c) * 2 + k];
            const double hk = E.h[s0 + k];
            const double N = st(k, l0, 0);
            const double dN = N + mp[3], dI = I + mp[4];
            const double lim = (N * I) / (dN * dI);
            const double b0 = qb(k, l0, 0);
            double limb = 0.0;
            if (model == M3D_MODEL_N) {
                const double fb = -b0 + Eb * hk;
                gv[2] += fb * lim;
                limb = fb * mp[2];
            } else if (model == M3D_MODEL_NDOP) {
                const double b1 = qb(k, l0, 1), DOP = st(k, l0, 1);
                const double f = mp[2] * lim;
                const double fb = -b0 + mp[5] * b1 + Eb * mp[7] * hk;
                gv[5] += b1 * f;
                gv[7] += Eb * f * hk;
                addy(k, l0, 1, mp[6] * (b0 - b1));
                gv[6] += (b0 - b1) * DOP;
                gv[2] += fb * lim;
                limb = fb * mp[2];
            } else {
                const double b1 = qb(k, l0, 1), b2 = qb(k, l0, 2);
                const double DOP = st(k, l0, 1), PHY = st(k, l0, 2);
                const double f1 = mp[2] * PHY * lim, f3 = mp[10] * f1;
                const double f3b = mp[6] * b1 + Eb * mp[12] * hk;
                gv[6] += b1 * f3;
                gv[12] += Eb * f3 * hk;
                const double f1b = -b0 + mp[11] * b2 + mp[10] * f3b;
                gv[10] += f3b * f1;
                gv[11] += b2 * f1;
                const double lossb = b1 - b2;
                addy(k, l0, 2, lossb * (mp[7] + 2.0 * mp[8] * PHY) + mp[9] * (b1 - b2) + f1b * mp[2] * lim);
                gv[7] += lossb * PHY;
                gv[8] += lossb * PHY * PHY;
                gv[9] += (b1 - b2) * PHY;
                addy(k, l0, 1, mp[5] * (b0 - b1));
                gv[5] += (b0 - b1) * DOP;
                gv[2] += f1b * PHY * lim;
                limb = f1b * mp[2] * PHY;
            }
            // lim = N I / ((N + K) (I + K_I))
            addy(k, l0, 0, limb * I * mp[3] / (dN * dN * dI));
            gv[3] += -limb * lim / dN;
            gv[4] += -limb * lim / dI;
            gv[0] += limb * (N * mp[4] / (dN * dI * dI)) * (-zc[s0 + k] * I);
        }
        add_member_gradients(ub, gv, 13, ml, E.mem_pidx[mi], lane);
    }
    __syncwarp();
}

// ybar_j = A_j^T zbar_j + ds (dq/dy)^T zbar_j on every (column, group) item, the parameter
// gradient into the block's accumulators and, at the end, into the block's own partial sums.
// X: the forward state y_j, packed.
__global__ void __launch_bounds__(kMaxWarps * kLanes) k_ens_adj_explicit(EnsParams E, EnsAdjParams A, int j,
                                                                         const double *__restrict__ X,
                                                                         const double *__restrict__ Zb,
                                                                         double *__restrict__ Yb)
{
    extern __shared__ double smem[];
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = blockIdx.x * E.cpb, c1 = min(c0 + E.cpb, E.ncol);
    const int cell0 = E.col_start[c0], cell1 = E.col_start[c1];
    const int p0 = E.rowptr[cell0], p1 = E.rowptr[cell1];
    const int zm = E.zmax;
    double *sval = smem;
    double *ub = sval + E.nnz_blk_max;                                    // [nmember][kParSlots]
    double *wb = ub + (size_t)A.nmember * kParSlots + (size_t)warp * (3 * zm * kLanes + 2 * kLanes);
    double *ys = wb, *zbs = ys + zm * kLanes, *ybs = zbs + zm * kLanes;
    double *Es = ybs + zm * kLanes, *Ebs = Es + kLanes;
    int *scol = (int *)(ub + (size_t)A.nmember * kParSlots + (size_t)nw * (3 * zm * kLanes + 2 * kLanes));
    int *counter = scol + E.nnz_blk_max;
    const int m0 = E.m0tab[j];
    const double w = E.wtab[j];
    {
        const double *a0 = A.eat + (size_t)m0 * E.e_mstride, *d0 = A.edt + (size_t)m0 * E.e_mstride;
        for (int p = threadIdx.x; p < p1 - p0; p += blockDim.x) {
            sval[p] = fma(w, d0[p0 + p], a0[p0 + p]);
            scol[p] = E.colidx[p0 + p];
        }
        for (int i = threadIdx.x; i < A.nmember * kParSlots; i += blockDim.x) ub[i] = 0.0;
        if (threadIdx.x == 0) *counter = 0;
    }
    __syncthreads();
    const int nitems = (c1 - c0) * E.ngroup;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(counter, 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= nitems) break;
        const int c = c0 + item / E.ngroup, g = item - (item / E.ngroup) * E.ngroup;
        const int s0 = E.col_start[c], L = E.col_start[c + 1] - s0;
        const size_t gl = (size_t)g * kLanes + lane;
        for (int k = 0; k < L; k++) {
            ys[k * kLanes + lane] = X[(size_t)(s0 + k) * E.wp + gl];
            zbs[k * kLanes + lane] = Zb[(size_t)(s0 + k) * E.wp + gl];
            const int pb = E.rowptr[s0 + k] - p0, pe = E.rowptr[s0 + k + 1] - p0;
            double z = 0.0;
            for (int p = pb; p < pe; p++) z = fma(sval[p], Zb[(size_t)scol[p] * E.wp + gl], z);
            ybs[k * kLanes + lane] = z;
        }
        __syncwarp();
        const double I0 = E.I0tab[(size_t)j * E.nulat + E.col_ulat[c]];
        for (int sg = E.grp_seg_off[g]; sg < E.grp_seg_off[g + 1]; sg++)
            ens_segment_qadj(E, A, E.segs[sg], c, s0, L, I0, lane, ys, zbs, ybs, Es, Ebs, ub);
        __syncwarp();
        for (int k = 0; k < L; k++) Yb[(size_t)(s0 + k) * E.wp + gl] = ybs[k * kLanes + lane];
        __syncwarp();
    }
    __syncthreads();
    double *part = A.ub_part + (size_t)blockIdx.x * A.nmember * kParSlots;
    for (int i = threadIdx.x; i < A.nmember * kParSlots; i += blockDim.x) part[i] += ub[i];
}

__host__ __device__ inline size_t ens_adj_smem_bytes(int nnz_blk_max, int zmax, int nwarps, int nmember)
{
    return sizeof(double) * ((size_t)nnz_blk_max + (size_t)nmember * kParSlots +
                             (size_t)nwarps * (3 * (size_t)zmax * kLanes + 2 * kLanes)) +
           sizeof(int) * ((size_t)nnz_blk_max + 4);
}

// out[m][p] = in[m][sym[p]]: the transposed matrix's values in the pattern's own slots.
__global__ void k_ens_transpose_values(long long nnz, int nmonth, const int *sym, const double *in, double *out)
{
    const long long tot = nnz * nmonth;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const long long m = i / nnz, p = i - m * nnz;
        out[i] = in[m * nnz + sym[p]];
    }
}

// ubar[m][q] = sum over blocks of part[b][m][q] (fixed order).
__global__ void k_ens_ubar_reduce(int nblocks, int nm, const double *part, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nm * kParSlots) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; b++) s += part[(size_t)b * nm * kParSlots + i];
    out[i] = s;
}

// Per-member tables from the derived scalars: light attenuation of the euphotic cells and the
// Martin deposition profile (F(z_top) - F(z_bot)) / (E h) of the aphotic cells, with the
// sea-floor rule (nothing leaves the bottom interface; a column without aphotic layers keeps
// its export in its bottom layer, 1/h there).
__global__ void k_ens_tables(int nmember, int ncol, int n, const int *col_start, const double *h,
                             const double *zc, const int *mem_model, const double *mpar, double *atten,
                             double *mfrac, double *mfrac_b)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nmember * ncol) return;
    const int m = (int)(idx / ncol), c = (int)(idx % ncol);
    const int model = mem_model[m];
    const double kw = mpar[(size_t)m * kParSlots + 0], b = mpar[(size_t)m * kParSlots + 1];
    const int s0 = col_start[c], L = col_start[c + 1] - s0, neu = L < 2 ? L : 2;
    for (int k = 0; k < 2; k++)
        atten[((size_t)m * ncol + c) * 2 + k] = k < neu ? kSigmaPar * exp(-kw * zc[s0 + k]) : 0.0;
    if (model == M3D_MODEL_NPZD) return;
    double zeu = 0.0;
    for (int k = 0; k < neu; k++) zeu += h[s0 + k];
    for (int k = 0; k < neu; k++) {
        mfrac[(size_t)m * n + s0 + k] = (L <= 2 && k == L - 1) ? 1.0 / h[s0 + k] : 0.0;
        if (mfrac_b) mfrac_b[(size_t)m * n + s0 + k] = 0.0;
    }
    double ztop = zeu;
    for (int k = neu; k < L; k++) {
        const double zbot = ztop + h[s0 + k];
        const double top = pow(ztop / zeu, -b);
        const double bot = k + 1 < L ? pow(zbot / zeu, -b) : 0.0;
        mfrac[(size_t)m * n + s0 + k] = (top - bot) / h[s0 + k];
        // d mfrac / d b, for the reverse sweep: d (z/z_eu)^-b / d b = -ln(z/z_eu) (z/z_eu)^-b
        if (mfrac_b) {
            const double dtop = -log(ztop / zeu) * top;
            const double dbot = k + 1 < L ? -log(zbot / zeu) * bot : 0.0;
            mfrac_b[(size_t)m * n + s0 + k] = (dtop - dbot) / h[s0 + k];
        }
        ztop = zbot;
    }
}

// [W][n] (members' rows) <-> X[n][wp] (cell-major, packed lanes; empty lanes zero).
__global__ void k_ens_pack(int n, int wp, const int *lane_tracer, const double *Y, double *X)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * wp) return;
    const int i = (int)(idx / wp), l = (int)(idx % wp), t = lane_tracer[l];
    X[idx] = t >= 0 ? Y[(size_t)t * n + i] : 0.0;
}
__global__ void k_ens_unpack(int n, int width, const int *tracer_lane, const double *X, int wp, double *Y)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * width) return;
    const int t = (int)(idx / n), i = (int)(idx % n);
    Y[idx] = X[(size_t)i * wp + tracer_lane[t]];
}

__global__ void k_ens_insolation(int nstep, int nulat, const double *ulat, double *I0)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nstep * nulat) return;
    const int jj = (int)(i / nulat), l = (int)(i % nulat);
    I0[i] = m3d::insolation(ulat[l], (double)jj / nstep);
}

thread_local std::string g_ens_init_error;

int model_ntracer(int model)
{
    switch (model) {
    case M3D_MODEL_N: return 1;
    case M3D_MODEL_NDOP: return 2;
    case M3D_MODEL_PHY: return 3;
    case M3D_MODEL_NPZD: return 5;
    default: return 0;
    }
}
int model_nparam(int model)
{
    switch (model) {
    case M3D_MODEL_N: return 5;
    case M3D_MODEL_NDOP: return 7;
    case M3D_MODEL_PHY: return 11;
    case M3D_MODEL_NPZD: return 13;
    default: return -1;
    }
}

// Derived scalars of one member (slot layout above).
void derive_params(int model, const double *u, double *mp)
{
    for (int i = 0; i < kParSlots; i++) mp[i] = 0.0;
    switch (model) {
    case M3D_MODEL_N:
        mp[0] = u[0]; mp[1] = u[4]; mp[2] = u[1] * 360.0; mp[3] = u[2]; mp[4] = u[3];
        break;
    case M3D_MODEL_NDOP:
        mp[0] = u[0]; mp[1] = u[6]; mp[2] = u[1] * 360.0; mp[3] = u[4]; mp[4] = u[5];
        mp[5] = u[2]; mp[6] = u[3]; mp[7] = 1.0 - u[2];
        break;
    case M3D_MODEL_PHY:
        mp[0] = u[1]; mp[1] = u[10]; mp[2] = 360.0 * u[0]; mp[3] = u[2]; mp[4] = u[3];
        mp[5] = 360.0 * u[4]; mp[6] = u[5]; mp[7] = 360.0 * u[6]; mp[8] = 360.0 * u[7]; mp[9] = 360.0 * u[8];
        mp[10] = u[9]; mp[11] = 1.0 - u[9]; mp[12] = 1.0 - u[5];
        break;
    case M3D_MODEL_NPZD:
        mp[0] = u[0]; mp[1] = 0.0; mp[2] = 360.0 * u[1]; mp[3] = u[2]; mp[4] = u[3];
        mp[5] = 360.0 * u[4]; mp[6] = u[5]; mp[7] = u[6]; mp[8] = 360.0 * u[7]; mp[9] = 360.0 * u[8];
        mp[10] = 360.0 * u[9]; mp[11] = 360.0 * u[10]; mp[12] = 360.0 * u[11]; mp[13] = 360.0 * u[12];
        mp[14] = 1.0 - u[6];
        break;
    }
}

}  // namespace

struct m3d_ensemble {
    int device = 0;
    cudaStream_t stream = nullptr;
    int n = 0, ncol = 0, nstep = 0, nmonth = 0, nsub = 1, nmember = 0, width = 0, ngroup = 0, wp = 0, zmax = 0;
    int cpb = 0, nwarps = 0, nblocks = 0;
    int tangent = 0;                           // members carry a perturbation (tangent ensembles)
    size_t smem = 0, smem_optin = 0;
    std::vector<int> col_start;
    std::vector<int> rowptr;
    std::vector<int> models, offsets;          // per member (offsets: nmember + 1)
    std::vector<double> u_host;                // [nmember][16] user parameters (copied)
    std::vector<double> mpar_host;             // [nmember][kParSlots]
    std::vector<void *> allocs;
    EnsParams P{};
    int *mem_model_dev = nullptr;
    double *mpar_dev = nullptr, *atten_dev = nullptr, *mfrac_dev = nullptr;
    int *lane_tracer = nullptr, *tracer_lane = nullptr;
    double *xbuf[2] = {nullptr, nullptr};
    // the reverse sweep (non-tangent ensembles whose explicit pattern is structurally
    // symmetric): transposed operators, d mfrac / d b, the members' parameter counts
    int adj_ok = 0;
    double *eat = nullptr, *edt = nullptr, *trit = nullptr, *mfrac_b_dev = nullptr;
    std::vector<int> nparams;
    cudaGraphExec_t graph = nullptr;
    long long last_launches = 0;
    std::string err;
};

namespace {

m3d_status efail(m3d_ensemble *e, m3d_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (e) e->err = buf;
    else g_ens_init_error = buf;
    return s;
}

#define ENS_CUDA(e, call)                                                                     \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return efail((e), M3D_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

template <typename T>
cudaError_t ens_upload(m3d_ensemble *e, T **dst, const T *src, size_t count)
{
    *dst = nullptr;
    if (count == 0) count = 1;
    cudaError_t r = cudaMalloc((void **)dst, sizeof(T) * count);
    if (r != cudaSuccess) return r;
    e->allocs.push_back(*dst);
    if (src) return cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice);
    return cudaSuccess;
}

void ens_release(m3d_ensemble *e)
{
    if (!e) return;
    if (e->graph) cudaGraphExecDestroy(e->graph);
    e->graph = nullptr;
    for (void *p : e->allocs) cudaFree(p);
    e->allocs.clear();
}

// Block sizes for cpb columns per block: largest entry and cell counts of a block.
void block_extents(const m3d_ensemble *e, int cpb, int *nnz_max, int *cells_max, int *nblocks)
{
    int nb = (e->ncol + cpb - 1) / cpb, a = 0, b = 0;
    for (int blk = 0; blk < nb; blk++) {
        int c0 = blk * cpb, c1 = std::min(c0 + cpb, e->ncol);
        int s = e->col_start[c0], t = e->col_start[c1];
        a = std::max(a, e->rowptr[t] - e->rowptr[s]);
        b = std::max(b, t - s);
    }
    *nnz_max = a;
    *cells_max = b;
    *nblocks = nb;
}

m3d_status apply_tiling(m3d_ensemble *e, int cpb, int nwarps)
{
    if (cpb < 1 || cpb > e->ncol || nwarps < 1 || nwarps > kMaxWarps)
        return efail(e, M3D_ERR_ARG, "tiling: columns per block must be 1..%d and warps 1..%d", e->ncol, kMaxWarps);
    int nnz_max, cells_max, nb;
    block_extents(e, cpb, &nnz_max, &cells_max, &nb);
    const bool sub1 = e->nsub == 1;
    size_t smem = ens_smem_bytes(nnz_max, cells_max, e->zmax, nwarps, sub1);
    if (smem > e->smem_optin)
        return efail(e, M3D_ERR_ARG, "tiling: %d columns x %d warps needs %zu bytes of shared memory (%zu available)",
                     cpb, nwarps, smem, e->smem_optin);
    const void *fn = sub1 ? (const void *)k_ens_step<true> : (const void *)k_ens_step<false>;
    ENS_CUDA(e, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    e->cpb = cpb;
    e->nwarps = nwarps;
    e->nblocks = nb;
    e->smem = smem;
    e->P.cpb = cpb;
    e->P.nnz_blk_max = nnz_max;
    e->P.cells_blk_max = cells_max;
    if (e->graph) {
        cudaGraphExecDestroy(e->graph);
        e->graph = nullptr;
    }
    return M3D_OK;
}

m3d_status launch_step(m3d_ensemble *e, int j, const double *X, double *Xn)
{
    if (e->nsub == 1)
        k_ens_step<true><<<e->nblocks, e->nwarps * kLanes, e->smem, e->stream>>>(e->P, j, X, Xn);
    else
        k_ens_step<false><<<e->nblocks, e->nwarps * kLanes, e->smem, e->stream>>>(e->P, j, X, Xn);
    ENS_CUDA(e, cudaGetLastError());
    return M3D_OK;
}

m3d_status launch_tables(m3d_ensemble *e)
{
    long long tot = (long long)e->nmember * e->ncol;
    k_ens_tables<<<(unsigned)((tot + 255) / 256), 256, 0, e->stream>>>(
        e->nmember, e->ncol, e->n, e->P.col_start, e->P.h, e->P.h + e->n, e->mem_model_dev, e->mpar_dev, e->atten_dev,
        e->mfrac_dev, e->mfrac_b_dev);
    ENS_CUDA(e, cudaGetLastError());
    return M3D_OK;
}

m3d_status pack(m3d_ensemble *e, const double *Y, double *X)
{
    long long tot = (long long)e->n * e->wp;
    k_ens_pack<<<(unsigned)((tot + 255) / 256), 256, 0, e->stream>>>(e->n, e->wp, e->lane_tracer, Y, X);
    ENS_CUDA(e, cudaGetLastError());
    return M3D_OK;
}

m3d_status unpack(m3d_ensemble *e, const double *X, double *Y)
{
    long long tot = (long long)e->n * e->width;
    k_ens_unpack<<<(unsigned)((tot + 255) / 256), 256, 0, e->stream>>>(e->n, e->width, e->tracer_lane, X, e->wp, Y);
    ENS_CUDA(e, cudaGetLastError());
    return M3D_OK;
}

m3d_status build_graph(m3d_ensemble *e)
{
    cudaStream_t s = e->stream;
    bool own = false;
    if (!s) {
        ENS_CUDA(e, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        own = true;
    }
    cudaStream_t saved = e->stream;
    e->stream = s;
    cudaGraph_t graph = nullptr;
    cudaError_t r = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    m3d_status st = M3D_OK;
    if (r == cudaSuccess) {
        for (int j = 0; j < e->nstep && st == M3D_OK; j++) st = launch_step(e, j, e->xbuf[j & 1], e->xbuf[(j + 1) & 1]);
        r = cudaStreamEndCapture(s, &graph);
    }
    e->stream = saved;
    if (own) cudaStreamDestroy(s);
    if (st != M3D_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (r != cudaSuccess) return efail(e, M3D_ERR_CUDA, "ensemble year graph capture: %s", cudaGetErrorString(r));
    r = cudaGraphInstantiate(&e->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (r != cudaSuccess) return efail(e, M3D_ERR_CUDA, "ensemble year graph instantiate: %s", cudaGetErrorString(r));
    return M3D_OK;
}

m3d_status upload_params(m3d_ensemble *e)
{
    ENS_CUDA(e, cudaMemcpyAsync(e->mpar_dev, e->mpar_host.data(), sizeof(double) * e->mpar_host.size(),
                                cudaMemcpyHostToDevice, e->stream));
    m3d_status st = launch_tables(e);
    if (st != M3D_OK) return st;
    ENS_CUDA(e, cudaStreamSynchronize(e->stream));
    return M3D_OK;
}

}  // namespace

m3d_status ensemble_init(m3d_ensemble **out, const m3d_grid *g, const m3d_matrices *mt, int nmember,
                         const m3d_member *members, int nsub, int nstep, void *stream, bool tangent);

extern "C" {

m3d_status metos3d_ensemble_init(m3d_ensemble **out, const m3d_grid *g, const m3d_matrices *mt, int nmember,
                                 const m3d_member *members, int nsub, int nstep, void *stream)
{
    return ensemble_init(out, g, mt, nmember, members, nsub, nstep, stream, false);
}

m3d_status metos3d_ensemble_init_tangent(m3d_ensemble **out, const m3d_grid *g, const m3d_matrices *mt, int nmember,
                                         const m3d_member *members, int nsub, int nstep, void *stream)
{
    return ensemble_init(out, g, mt, nmember, members, nsub, nstep, stream, true);
}

}  // extern "C"

m3d_status ensemble_init(m3d_ensemble **out, const m3d_grid *g, const m3d_matrices *mt, int nmember,
                         const m3d_member *members, int nsub, int nstep, void *stream, bool tangent)
{
    if (!out) return efail(nullptr, M3D_ERR_ARG, "metos3d_ensemble_init: out is null");
    *out = nullptr;
    std::string why;
    if (m3d_validate_inputs(g, mt, why) != M3D_OK) return efail(nullptr, M3D_ERR_ARG, "%s", why.c_str());
    if (nmember < 1 || nmember > 4096 || !members)
        return efail(nullptr, M3D_ERR_ARG, "ensemble: 1..4096 members needed");
    if (nsub < 1 || nstep < 1) return efail(nullptr, M3D_ERR_ARG, "ensemble: nsub and nstep must be positive");
    for (int m = 0; m < nmember; m++) {
        const int model = members[m].model_id;
        if (model_ntracer(model) == 0)
            return efail(nullptr, M3D_ERR_UNSUPPORTED, "ensemble: member %d has unknown model %d", m, model);
        if (members[m].nparam != model_nparam(model) || !members[m].u)
            return efail(nullptr, M3D_ERR_ARG, "ensemble: member %d needs %d parameters", m, model_nparam(model));
        for (int i = 0; i < members[m].nparam; i++)
            if (!std::isfinite(members[m].u[i]))
                return efail(nullptr, M3D_ERR_ARG, "ensemble: member %d has a non-finite parameter", m);
    }
    m3d_ensemble *e = new (std::nothrow) m3d_ensemble();
    if (!e) return efail(nullptr, M3D_ERR_ARG, "out of host memory");
    auto bail = [&](m3d_status s) {
        g_ens_init_error = e->err;
        ens_release(e);
        delete e;
        return s;
    };
#define ENS_UP(call)                                                                              \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            efail(e, M3D_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));               \
            return bail(M3D_ERR_CUDA);                                                            \
        }                                                                                         \
    } while (0)
    cudaGetDevice(&e->device);
    e->stream = (cudaStream_t)stream;
    e->n = g->n;
    e->ncol = g->ncol;
    e->nstep = nstep;
    e->nmonth = mt->nmonth;
    e->nsub = nsub;
    e->nmember = nmember;
    e->tangent = tangent ? 1 : 0;
    const int lanes_per_tracer = tangent ? 2 : 1;
    e->col_start.assign(g->col_start, g->col_start + g->ncol + 1);
    e->rowptr.assign(mt->exp_rowptr, mt->exp_rowptr + g->n + 1);
    for (int c = 0; c < g->ncol; c++) e->zmax = std::max(e->zmax, g->col_start[c + 1] - g->col_start[c]);

    // ---- members: tracer offsets, packing into 32-lane groups (more tracers first, first fit)
    e->models.resize(nmember);
    e->offsets.assign(nmember + 1, 0);
    e->mpar_host.assign((size_t)nmember * kParSlots, 0.0);
    for (int m = 0; m < nmember; m++) {
        e->models[m] = members[m].model_id;
        e->offsets[m + 1] = e->offsets[m] + model_ntracer(members[m].model_id);
        derive_params(members[m].model_id, members[m].u, &e->mpar_host[(size_t)m * kParSlots]);
    }
    const int W = e->offsets[nmember];
    e->width = lanes_per_tracer * W;
    std::vector<int> order(nmember);
    for (int m = 0; m < nmember; m++) order[m] = m;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return model_ntracer(e->models[a]) > model_ntracer(e->models[b]); });
    std::vector<int> fill;                       // lanes used per group
    std::vector<int> grp(nmember), lane0(nmember);
    for (int m : order) {
        int nt = lanes_per_tracer * model_ntracer(e->models[m]), gsel = -1;
        for (int gi = 0; gi < (int)fill.size() && gsel < 0; gi++)
            if (fill[gi] + nt <= kLanes) gsel = gi;
        if (gsel < 0) {
            gsel = (int)fill.size();
            fill.push_back(0);
        }
        grp[m] = gsel;
        lane0[m] = fill[gsel];
        fill[gsel] += nt;
    }
    e->ngroup = (int)fill.size();
    e->wp = e->ngroup * kLanes;
    // member slots grouped by group, then by model; one segment per (group, model)
    std::vector<int> slots(nmember);
    for (int m = 0; m < nmember; m++) slots[m] = m;
    std::stable_sort(slots.begin(), slots.end(), [&](int a, int b) {
        if (grp[a] != grp[b]) return grp[a] < grp[b];
        return e->models[a] < e->models[b];
    });
    std::vector<int> mem_lane0(nmember), mem_pidx(nmember), seg_off(e->ngroup + 1, 0);
    std::vector<int4> segs;
    for (int s = 0; s < nmember; s++) {
        int m = slots[s];
        mem_lane0[s] = lane0[m];
        mem_pidx[s] = m;
        if (s == 0 || grp[slots[s - 1]] != grp[m] || e->models[slots[s - 1]] != e->models[m])
            segs.push_back(make_int4(e->models[m], s, s, e->tangent));
        segs.back().z = s + 1;
        seg_off[grp[m] + 1] = (int)segs.size();
    }
    for (int gi = 1; gi <= e->ngroup; gi++) seg_off[gi] = std::max(seg_off[gi], seg_off[gi - 1]);
    std::vector<int> lane_tracer(e->wp, -1), tracer_lane(e->width);
    for (int m = 0; m < nmember; m++) {
        const int nt = model_ntracer(e->models[m]);
        for (int t = 0; t < nt; t++) {
            int l = grp[m] * kLanes + lane0[m] + t;
            lane_tracer[l] = e->offsets[m] + t;
            tracer_lane[e->offsets[m] + t] = l;
            if (tangent) {                    // the perturbation: nt lanes on, rows W on
                lane_tracer[l + nt] = W + e->offsets[m] + t;
                tracer_lane[W + e->offsets[m] + t] = l + nt;
            }
        }
    }

    // ---- Thomas factors of every monthly implicit block (required)
    std::vector<double> tri((size_t)mt->nmonth * 3 * g->n);
    {
        std::vector<long long> blk_off(g->ncol + 1, 0);
        for (int c = 0; c < g->ncol; c++) {
            long long L = g->col_start[c + 1] - g->col_start[c];
            blk_off[c + 1] = blk_off[c] + L * L;
        }
        for (int m = 0; m < mt->nmonth; m++)
            for (int c = 0; c < g->ncol; c++) {
                int L = g->col_start[c + 1] - g->col_start[c], s0 = g->col_start[c];
                double *base = tri.data() + (size_t)m * 3 * g->n;
                if (!tridiagonal_factors(mt->imp_blk + (size_t)m * mt->s_imp + blk_off[c], L, base + s0,
                                         base + g->n + s0, base + 2 * (size_t)g->n + s0)) {
                    efail(e, M3D_ERR_UNSUPPORTED,
                          "ensemble: the implicit block of column %d, month %d is not the inverse of a tridiagonal matrix",
                          c, m);
                    return bail(M3D_ERR_UNSUPPORTED);
                }
            }
        for (int m = 0; m < mt->nmonth; m++)
            thomas_backsubstitution_form(tri.data() + (size_t)m * 3 * g->n, g->n, g->col_start, g->ncol);
    }
    // ---- explicit values and month differences
    const size_t nnz = (size_t)mt->nnz;
    std::vector<double> ed((size_t)mt->nmonth * nnz);
    for (int m = 0; m < mt->nmonth; m++) {
        const double *a = mt->exp_val + (size_t)m * nnz, *b = mt->exp_val + (size_t)((m + 1) % mt->nmonth) * nnz;
        for (size_t p = 0; p < nnz; p++) ed[(size_t)m * nnz + p] = b[p] - a[p];
    }
    // ---- step tables, latitudes
    std::vector<int> m0tab(nstep);
    std::vector<double> wtab(nstep);
    for (int j = 0; j < nstep; j++) m3d::month_weights(j, nstep, mt->nmonth, m0tab[j], wtab[j]);
    std::vector<double> ulat(g->lat, g->lat + g->ncol);
    std::sort(ulat.begin(), ulat.end());
    ulat.erase(std::unique(ulat.begin(), ulat.end()), ulat.end());
    std::vector<int> col_ulat(g->ncol);
    for (int c = 0; c < g->ncol; c++)
        col_ulat[c] = (int)(std::lower_bound(ulat.begin(), ulat.end(), g->lat[c]) - ulat.begin());

    cudaDeviceProp prop;
    ENS_UP(cudaGetDeviceProperties(&prop, e->device));
    e->smem_optin = prop.sharedMemPerBlockOptin;

    EnsParams &P = e->P;
    P.n = g->n;
    P.ncol = g->ncol;
    P.nstep = nstep;
    P.nmonth = mt->nmonth;
    P.nsub = nsub;
    P.wp = e->wp;
    P.ngroup = e->ngroup;
    P.nulat = (int)ulat.size();
    P.zmax = e->zmax;
    P.ds = (1.0 / nstep) / nsub;
    P.e_mstride = (long long)nnz;
    P.tri_mstride = 3LL * g->n;
    {
        int *ip;
        double *dp;
        ENS_UP(ens_upload(e, &ip, m0tab.data(), m0tab.size())); P.m0tab = ip;
        ENS_UP(ens_upload(e, &dp, wtab.data(), wtab.size())); P.wtab = dp;
        ENS_UP(ens_upload(e, &ip, mt->exp_rowptr, (size_t)g->n + 1)); P.rowptr = ip;
        ENS_UP(ens_upload(e, &ip, mt->exp_colidx, nnz)); P.colidx = ip;
        ENS_UP(ens_upload(e, &dp, mt->exp_val, (size_t)mt->nmonth * nnz)); P.ea = dp;
        ENS_UP(ens_upload(e, &dp, ed.data(), ed.size())); P.ed = dp;
        ENS_UP(ens_upload(e, &dp, tri.data(), tri.size())); P.tri = dp;
        ENS_UP(ens_upload(e, &ip, g->col_start, (size_t)g->ncol + 1)); P.col_start = ip;
        ENS_UP(ens_upload(e, &ip, col_ulat.data(), col_ulat.size())); P.col_ulat = ip;
        std::vector<double> hz(g->h, g->h + g->n);
        hz.insert(hz.end(), g->zc, g->zc + g->n);
        ENS_UP(ens_upload(e, &dp, hz.data(), hz.size())); P.h = dp;     // h, then zc
        double *ulat_dev, *I0;
        ENS_UP(ens_upload(e, &ulat_dev, ulat.data(), ulat.size()));
        ENS_UP(ens_upload(e, &I0, (const double *)nullptr, (size_t)nstep * ulat.size()));
        long long tot = (long long)nstep * (long long)ulat.size();
        k_ens_insolation<<<(unsigned)((tot + 255) / 256), 256>>>(nstep, (int)ulat.size(), ulat_dev, I0);
        ENS_UP(cudaGetLastError());
        P.I0tab = I0;
        ENS_UP(ens_upload(e, &ip, seg_off.data(), seg_off.size())); P.grp_seg_off = ip;
        int4 *sp;
        ENS_UP(ens_upload(e, &sp, segs.data(), segs.size())); P.segs = sp;
        ENS_UP(ens_upload(e, &ip, mem_lane0.data(), mem_lane0.size())); P.mem_lane0 = ip;
        ENS_UP(ens_upload(e, &ip, mem_pidx.data(), mem_pidx.size())); P.mem_pidx = ip;
        ENS_UP(ens_upload(e, &e->mem_model_dev, e->models.data(), e->models.size()));
        ENS_UP(ens_upload(e, &e->mpar_dev, e->mpar_host.data(), e->mpar_host.size())); P.mpar = e->mpar_dev;
        ENS_UP(ens_upload(e, &e->atten_dev, (const double *)nullptr, (size_t)nmember * g->ncol * 2)); P.atten = e->atten_dev;
        ENS_UP(ens_upload(e, &e->mfrac_dev, (const double *)nullptr, (size_t)nmember * g->n)); P.mfrac = e->mfrac_dev;
        ENS_UP(cudaMemset(e->mfrac_dev, 0, sizeof(double) * (size_t)nmember * g->n));
        ENS_UP(ens_upload(e, &e->lane_tracer, lane_tracer.data(), lane_tracer.size()));
        ENS_UP(ens_upload(e, &e->tracer_lane, tracer_lane.data(), tracer_lane.size()));
        double *xb;
        ENS_UP(ens_upload(e, &xb, (const double *)nullptr, 2 * (size_t)g->n * e->wp));
        ENS_UP(cudaMemset(xb, 0, sizeof(double) * 2 * (size_t)g->n * e->wp));
        e->xbuf[0] = xb;
        e->xbuf[1] = xb + (size_t)g->n * e->wp;
    }
    // ---- the reverse sweep's operators: A_m^T in the pattern's slots (a structurally
    // symmetric pattern holds the transpose's entries), Thomas factors of every T_m^T
    e->nparams.resize(nmember);
    for (int m = 0; m < nmember; m++) e->nparams[m] = model_nparam(e->models[m]);
    if (!tangent) {
        std::vector<int> sym(nnz);
        bool symmetric = true;
        for (int i = 0; i < g->n && symmetric; i++)
            for (int q = mt->exp_rowptr[i]; q < mt->exp_rowptr[i + 1] && symmetric; q++) {
                const int k = mt->exp_colidx[q];
                const int *b = mt->exp_colidx + mt->exp_rowptr[k], *en = mt->exp_colidx + mt->exp_rowptr[k + 1];
                const int *f = std::lower_bound(b, en, i);
                if (f == en || *f != i) symmetric = false;
                else sym[q] = (int)(f - mt->exp_colidx);
            }
        std::vector<double> trit;
        bool tri_t = symmetric;
        if (tri_t) {
            trit.assign((size_t)mt->nmonth * 3 * g->n, 0.0);
            std::vector<double> bt;
            long long off = 0;
            std::vector<long long> blk_off(g->ncol + 1, 0);
            for (int c = 0; c < g->ncol; c++) {
                long long L = g->col_start[c + 1] - g->col_start[c];
                blk_off[c + 1] = blk_off[c] + L * L;
            }
            (void)off;
            for (int m = 0; m < mt->nmonth && tri_t; m++) {
                double *base = trit.data() + (size_t)m * 3 * g->n;
                for (int c = 0; c < g->ncol && tri_t; c++) {
                    const int L = g->col_start[c + 1] - g->col_start[c], s0 = g->col_start[c];
                    const double *B = mt->imp_blk + (size_t)m * mt->s_imp + blk_off[c];
                    bt.assign((size_t)L * L, 0.0);
                    for (int r = 0; r < L; r++)
                        for (int k = 0; k < L; k++) bt[(size_t)k * L + r] = B[(size_t)r * L + k];
                    tri_t = tridiagonal_factors(bt.data(), L, base + s0, base + g->n + s0, base + 2 * (size_t)g->n + s0);
                }
            }
            for (int m = 0; m < mt->nmonth && tri_t; m++)
                thomas_backsubstitution_form(trit.data() + (size_t)m * 3 * g->n, g->n, g->col_start, g->ncol);
        }
        if (symmetric && tri_t) {
            int *sym_dev;
            ENS_UP(ens_upload(e, &sym_dev, sym.data(), sym.size()));
            ENS_UP(ens_upload(e, &e->eat, (const double *)nullptr, (size_t)mt->nmonth * nnz));
            ENS_UP(ens_upload(e, &e->edt, (const double *)nullptr, (size_t)mt->nmonth * nnz));
            k_ens_transpose_values<<<1024, 256>>>((long long)nnz, mt->nmonth, sym_dev, P.ea, e->eat);
            k_ens_transpose_values<<<1024, 256>>>((long long)nnz, mt->nmonth, sym_dev, P.ed, e->edt);
            ENS_UP(cudaGetLastError());
            ENS_UP(ens_upload(e, &e->trit, trit.data(), trit.size()));
            ENS_UP(ens_upload(e, &e->mfrac_b_dev, (const double *)nullptr, (size_t)nmember * g->n));
            ENS_UP(cudaMemset(e->mfrac_b_dev, 0, sizeof(double) * (size_t)nmember * g->n));
            e->adj_ok = 1;
        }
    }
    ENS_UP(cudaDeviceSynchronize());
    m3d_status st = upload_params(e);
    if (st != M3D_OK) return bail(st);
    // default tiling: 4 columns and 8 warps per block, or the largest that fits
    st = M3D_ERR_ARG;
    for (int cpb = 4; cpb >= 1 && st != M3D_OK; cpb /= 2)
        for (int nw = 8; nw >= 1 && st != M3D_OK; nw /= 2) st = apply_tiling(e, std::min(cpb, e->ncol), nw);
    if (st != M3D_OK) return bail(st);
    e->err.clear();
    *out = e;
    return M3D_OK;
#undef ENS_UP
}

extern "C" {

m3d_status metos3d_ensemble_layout(const m3d_ensemble *e, int *nmember, int *width, int *n, int *ngroup, int *offsets)
{
    if (!e) return efail(nullptr, M3D_ERR_ARG, "metos3d_ensemble_layout: null ensemble");
    if (nmember) *nmember = e->nmember;
    if (width) *width = e->width;
    if (n) *n = e->n;
    if (ngroup) *ngroup = e->ngroup;
    if (offsets) std::copy(e->offsets.begin(), e->offsets.end(), offsets);
    return M3D_OK;
}

m3d_status metos3d_ensemble_set_stream(m3d_ensemble *e, void *stream)
{
    if (!e) return efail(nullptr, M3D_ERR_ARG, "metos3d_ensemble_set_stream: null ensemble");
    e->stream = (cudaStream_t)stream;
    return M3D_OK;
}

m3d_status metos3d_ensemble_set_params(m3d_ensemble *e, int member, const double *u)
{
    if (!e) return efail(nullptr, M3D_ERR_ARG, "metos3d_ensemble_set_params: null ensemble");
    if (member < 0 || member >= e->nmember || !u) return efail(e, M3D_ERR_ARG, "set_params: bad member or null u");
    const int np = model_nparam(e->models[member]);
    for (int i = 0; i < np; i++)
        if (!std::isfinite(u[i])) return efail(e, M3D_ERR_ARG, "set_params: non-finite parameter");
    derive_params(e->models[member], u, &e->mpar_host[(size_t)member * kParSlots]);
    return upload_params(e);
}

m3d_status metos3d_ensemble_steps(m3d_ensemble *e, int j0, int nsteps, const double *Y0, double *Y1)
{
    if (!e) return efail(nullptr, M3D_ERR_ARG, "metos3d_ensemble_steps: null ensemble");
    if (!Y0 || !Y1 || nsteps < 0 || j0 < 0) return efail(e, M3D_ERR_ARG, "steps: null state or negative count");
    m3d_status st = pack(e, Y0, e->xbuf[0]);
    for (int s = 0; s < nsteps && st == M3D_OK; s++)
        st = launch_step(e, (int)(((long long)j0 + s) % e->nstep), e->xbuf[s & 1], e->xbuf[(s + 1) & 1]);
    if (st == M3D_OK) st = unpack(e, e->xbuf[nsteps & 1], Y1);
    e->last_launches = nsteps + 2;
    return st;
}

m3d_status metos3d_ensemble_year_map(m3d_ensemble *e, const double *Y0, double *Y1)
{
    if (!e) return efail(nullptr, M3D_ERR_ARG, "metos3d_ensemble_year_map: null ensemble");
    if (!Y0 || !Y1) return efail(e, M3D_ERR_ARG, "year_map: null state");
    if (!e->graph) {
        m3d_status st = build_graph(e);
        if (st != M3D_OK) return st;
    }
    m3d_status st = pack(e, Y0, e->xbuf[0]);
    if (st != M3D_OK) return st;
    ENS_CUDA(e, cudaGraphLaunch(e->graph, e->stream));
    st = unpack(e, e->xbuf[e->nstep & 1], Y1);
    e->last_launches = e->nstep + 2;
    return st;
}

m3d_status metos3d_ensemble_set_tiling(m3d_ensemble *e, int cpb, int nwarps)
{
    if (!e) return efail(nullptr, M3D_ERR_ARG, "metos3d_ensemble_set_tiling: null ensemble");
    return apply_tiling(e, cpb, nwarps);
}

m3d_status metos3d_ensemble_get_tiling(const m3d_ensemble *e, int *cpb, int *nwarps)
{
    if (!e) return efail(nullptr, M3D_ERR_ARG, "metos3d_ensemble_get_tiling: null ensemble");
    if (cpb) *cpb = e->cpb;
    if (nwarps) *nwarps = e->nwarps;
    return M3D_OK;
}

m3d_status metos3d_ensemble_autotune(m3d_ensemble *e, const double *Y, int nsteps, int *cpb_out, int *nw_out,
                                     double *ms_out)
{
    if (!e) return efail(nullptr, M3D_ERR_ARG, "metos3d_ensemble_autotune: null ensemble");
    if (!Y || nsteps < 1) return efail(e, M3D_ERR_ARG, "autotune: null state or no steps");
    const int cpbs[] = {1, 2, 4, 8, 16, 32};
    const int nws[] = {4, 5, 6, 8, 10, 12, 16};
    int best_c = e->cpb, best_w = e->nwarps;
    float best = -1.0f;
    cudaEvent_t a, b;
    ENS_CUDA(e, cudaEventCreate(&a));
    ENS_CUDA(e, cudaEventCreate(&b));
    m3d_status st = M3D_OK;
    for (int cpb : cpbs) {
        if (cpb > e->ncol) continue;
        for (int nw : nws) {
            if (apply_tiling(e, cpb, nw) != M3D_OK) continue;     // does not fit
            st = pack(e, Y, e->xbuf[0]);
            for (int s = 0; s < 2 && st == M3D_OK; s++) st = launch_step(e, s, e->xbuf[s & 1], e->xbuf[(s + 1) & 1]);
            if (st != M3D_OK) break;
            cudaEventRecord(a, e->stream);
            for (int s = 0; s < nsteps && st == M3D_OK; s++)
                st = launch_step(e, s, e->xbuf[s & 1], e->xbuf[(s + 1) & 1]);
            cudaEventRecord(b, e->stream);
            if (st != M3D_OK) break;
            if (cudaEventSynchronize(b) != cudaSuccess) { st = efail(e, M3D_ERR_CUDA, "autotune: timing failed"); break; }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, a, b);
            ms /= nsteps;
            if (best < 0.0f || ms < best) {
                best = ms;
                best_c = cpb;
                best_w = nw;
            }
        }
        if (st != M3D_OK) break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != M3D_OK) return st;
    if (best < 0.0f) return efail(e, M3D_ERR_ARG, "autotune: no tiling fits in shared memory");
    st = apply_tiling(e, best_c, best_w);
    if (st != M3D_OK) return st;
    if (cpb_out) *cpb_out = best_c;
    if (nw_out) *nw_out = best_w;
    if (ms_out) *ms_out = best;
    return M3D_OK;
}

// The gradient in the derived slots of one member (slot 0: d/dk_w, slot 1: d/db, the others
// d/dmp[s] of derive_params) to the gradient in the user's parameters (the chain rule of
// derive_params: the rates per day times 360, the complements 1 - sigma).
static void derived_to_user(int model, const double *g, double *ub)
{
    switch (model) {
    case M3D_MODEL_N:
        ub[0] = g[0]; ub[1] = 360.0 * g[2]; ub[2] = g[3]; ub[3] = g[4]; ub[4] = g[1];
        break;
    case M3D_MODEL_NDOP:
        ub[0] = g[0]; ub[1] = 360.0 * g[2]; ub[2] = g[5] - g[7]; ub[3] = g[6]; ub[4] = g[3]; ub[5] = g[4];
        ub[6] = g[1];
        break;
    case M3D_MODEL_PHY:
        ub[0] = 360.0 * g[2]; ub[1] = g[0]; ub[2] = g[3]; ub[3] = g[4]; ub[4] = 360.0 * g[5]; ub[5] = g[6] - g[12];
        ub[6] = 360.0 * g[7]; ub[7] = 360.0 * g[8]; ub[8] = 360.0 * g[9]; ub[9] = g[10] - g[11]; ub[10] = g[1];
        break;
    case M3D_MODEL_NPZD:
        ub[0] = g[0]; ub[1] = 360.0 * g[2]; ub[2] = g[3]; ub[3] = g[4]; ub[4] = 360.0 * g[5]; ub[5] = g[6];
        ub[6] = g[7] - g[14]; ub[7] = 360.0 * g[8]; ub[8] = 360.0 * g[9]; ub[9] = 360.0 * g[10];
        ub[10] = 360.0 * g[11]; ub[11] = 360.0 * g[12]; ub[12] = 360.0 * g[13];
        break;
    }
}

m3d_status metos3d_ensemble_year_adjoint(m3d_ensemble *e, const double *Y0, const double *Ybar1, double *Ybar0,
                                         double *ubar_host, int ckpt_every)
{
    if (!e) return efail(nullptr, M3D_ERR_ARG, "metos3d_ensemble_year_adjoint: null ensemble");
    if (!Y0 || !Ybar1 || !Ybar0) return efail(e, M3D_ERR_ARG, "year_adjoint: null state");
    if (!e->adj_ok)
        return efail(e, M3D_ERR_UNSUPPORTED, "year_adjoint: needs a plain (not tangent) ensemble whose explicit "
                                             "pattern is structurally symmetric");
    if (e->nsub != 1) return efail(e, M3D_ERR_UNSUPPORTED, "year_adjoint: one internal model step only");
    const size_t smem_adj = ens_adj_smem_bytes(e->P.nnz_blk_max, e->zmax, e->nwarps, e->nmember);
    if (smem_adj > e->smem_optin)
        return efail(e, M3D_ERR_UNSUPPORTED, "year_adjoint: %zu bytes of shared memory needed (%zu available); "
                                             "choose a smaller tiling", smem_adj, e->smem_optin);
    ENS_CUDA(e, cudaFuncSetAttribute((const void *)k_ens_adj_explicit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_adj));
    const size_t smem_imp = sizeof(double) * (6 * (size_t)e->P.cells_blk_max + (size_t)e->nwarps * 2 * e->zmax * kLanes) +
                            sizeof(int) * 4;
    ENS_CUDA(e, cudaFuncSetAttribute((const void *)k_ens_adj_implicit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_imp));
    const int nstep = e->nstep;
    const int K = ckpt_every <= 0 ? 240 : std::min(ckpt_every, nstep);
    const int nseg = (nstep + K - 1) / K;
    const size_t state = sizeof(double) * (size_t)e->n * e->wp;
    // within a segment the states are kept every K2 steps and each K2-step piece recomputed
    // in full before its reverse steps: K2 = K unless K states would take more than half of
    // the free device memory (two levels of checkpoints, each step recomputed at most twice)
    size_t free_b = 0, total_b = 0;
    ENS_CUDA(e, cudaMemGetInfo(&free_b, &total_b));
    const size_t budget = free_b / 2 > (size_t)nseg * state ? free_b / 2 - (size_t)nseg * state : 0;
    long long K2 = std::min<long long>(K, (long long)(budget / state) / 2);
    if (K2 < 1) return efail(e, M3D_ERR_CUDA, "year_adjoint: not enough device memory for the checkpoints");
    const int nsub_max = (int)((K + K2 - 1) / K2);
    double *chk = nullptr, *sub = nullptr, *traj = nullptr, *ybw = nullptr, *zb = nullptr, *upart = nullptr, *ured = nullptr;
    auto cleanup = [&]() {
        for (double *q : {chk, sub, traj, ybw, zb, upart, ured})
            if (q) cudaFree(q);
    };
    cudaError_t r = cudaMalloc(&chk, state * nseg);
    if (r == cudaSuccess) r = cudaMalloc(&sub, state * nsub_max);
    if (r == cudaSuccess) r = cudaMalloc(&traj, state * K2);
    if (r == cudaSuccess) r = cudaMalloc(&ybw, 2 * state);
    if (r == cudaSuccess) r = cudaMalloc(&zb, state);
    if (r == cudaSuccess) r = cudaMalloc(&upart, sizeof(double) * (size_t)e->nblocks * e->nmember * kParSlots);
    if (r == cudaSuccess) r = cudaMalloc(&ured, sizeof(double) * (size_t)e->nmember * kParSlots);
    if (r != cudaSuccess) {
        cleanup();
        return efail(e, M3D_ERR_CUDA, "year_adjoint: %s", cudaGetErrorString(r));
    }
    EnsAdjParams A{e->eat, e->edt, e->trit, e->mfrac_b_dev, upart, e->nmember};
    long long launches = 0;
    auto run = [&]() -> m3d_status {
        ENS_CUDA(e, cudaMemsetAsync(upart, 0, sizeof(double) * (size_t)e->nblocks * e->nmember * kParSlots, e->stream));
        ENS_CUDA(e, cudaMemsetAsync(ybw, 0, 2 * state, e->stream));
        ENS_CUDA(e, cudaMemsetAsync(zb, 0, state, e->stream));
        // forward sweep: a checkpoint at the start of every segment
        m3d_status st = pack(e, Y0, chk);
        launches++;
        for (int sg = 0; sg + 1 < nseg && st == M3D_OK; sg++) {
            double *a = chk + (size_t)sg * e->n * e->wp, *b = chk + (size_t)(sg + 1) * e->n * e->wp;
            for (int jj = sg * K; jj < (sg + 1) * K && st == M3D_OK; jj++) {
                const int s = jj - sg * K;
                const double *in = s == 0 ? a : e->xbuf[s & 1];
                double *out = jj + 1 == (sg + 1) * K ? b : e->xbuf[(s + 1) & 1];
                st = launch_step(e, jj, in, out);
                launches++;
            }
        }
        if (st != M3D_OK) return st;
        st = pack(e, Ybar1, ybw);
        launches++;
        int cur = 0;
        for (int sg = nseg - 1; sg >= 0 && st == M3D_OK; sg--) {
            const int j0 = sg * K, j1 = std::min(j0 + K, nstep);
            const int nsub_seg = (int)((j1 - j0 + K2 - 1) / K2);
            // sub-checkpoints of the segment
            ENS_CUDA(e, cudaMemcpyAsync(sub, chk + (size_t)sg * e->n * e->wp, state, cudaMemcpyDeviceToDevice,
                                        e->stream));
            for (int q = 0; q + 1 < nsub_seg && st == M3D_OK; q++) {
                const int a0 = j0 + (int)(q * K2), a1 = j0 + (int)((q + 1) * K2);
                for (int jj = a0; jj < a1 && st == M3D_OK; jj++) {
                    const int s = jj - a0;
                    const double *in = s == 0 ? sub + (size_t)q * e->n * e->wp : e->xbuf[s & 1];
                    double *out = jj + 1 == a1 ? sub + (size_t)(q + 1) * e->n * e->wp : e->xbuf[(s + 1) & 1];
                    st = launch_step(e, jj, in, out);
                    launches++;
                }
            }
            for (int q = nsub_seg - 1; q >= 0 && st == M3D_OK; q--) {
                const int a0 = j0 + (int)(q * K2), a1 = std::min(j1, j0 + (int)((q + 1) * K2));
                ENS_CUDA(e, cudaMemcpyAsync(traj, sub + (size_t)q * e->n * e->wp, state, cudaMemcpyDeviceToDevice,
                                            e->stream));
                for (int jj = a0; jj + 1 < a1 && st == M3D_OK; jj++) {
                    st = launch_step(e, jj, traj + (size_t)(jj - a0) * e->n * e->wp,
                                     traj + (size_t)(jj - a0 + 1) * e->n * e->wp);
                    launches++;
                }
                for (int jj = a1 - 1; jj >= a0 && st == M3D_OK; jj--) {
                    double *yin = ybw + (size_t)cur * e->n * e->wp, *yout = ybw + (size_t)(1 - cur) * e->n * e->wp;
                    k_ens_adj_implicit<<<e->nblocks, e->nwarps * kLanes, smem_imp, e->stream>>>(e->P, A, jj, yin, zb);
                    k_ens_adj_explicit<<<e->nblocks, e->nwarps * kLanes, smem_adj, e->stream>>>(
                        e->P, A, jj, traj + (size_t)(jj - a0) * e->n * e->wp, zb, yout);
                    ENS_CUDA(e, cudaGetLastError());
                    launches += 2;
                    cur = 1 - cur;
                }
            }
        }
        if (st != M3D_OK) return st;
        st = unpack(e, ybw + (size_t)cur * e->n * e->wp, Ybar0);
        launches++;
        if (st != M3D_OK) return st;
        const int nm = e->nmember;
        k_ens_ubar_reduce<<<(nm * kParSlots + 127) / 128, 128, 0, e->stream>>>(e->nblocks, nm, upart, ured);
        ENS_CUDA(e, cudaGetLastError());
        launches++;
        std::vector<double> g((size_t)nm * kParSlots);
        ENS_CUDA(e, cudaMemcpyAsync(g.data(), ured, sizeof(double) * g.size(), cudaMemcpyDeviceToHost, e->stream));
        ENS_CUDA(e, cudaStreamSynchronize(e->stream));
        if (ubar_host) {
            size_t at = 0;
            for (int m = 0; m < nm; m++) {
                derived_to_user(e->models[m], g.data() + (size_t)m * kParSlots, ubar_host + at);
                at += (size_t)e->nparams[m];
            }
        }
        return M3D_OK;
    };
    m3d_status st = run();
    cudaStreamSynchronize(e->stream);
    cleanup();
    e->last_launches = launches;
    return st;
}

long long metos3d_ensemble_last_launch_count(const m3d_ensemble *e) { return e ? e->last_launches : -1; }

const char *metos3d_ensemble_last_error(const m3d_ensemble *e)
{
    return e ? e->err.c_str() : g_ens_init_error.c_str();
}

void metos3d_ensemble_free(m3d_ensemble *e)
{
    if (!e) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(e->device);
    ens_release(e);
    cudaSetDevice(cur);
    delete e;
}

}  // extern "C"
