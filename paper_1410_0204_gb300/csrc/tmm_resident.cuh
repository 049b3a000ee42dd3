// tmm_resident.cuh -- the year map (Metos3D, arXiv:1410.0204, Section 4) as one persistent
// launch whose tiles keep their month of transport matrices in shared memory.
//
// Within one month of the year (240 of the 2880 steps) a tile reads the same four arrays
// every step: A_m, A_{m+1} - A_m, B_m, B_{m+1} - B_m; only the interpolation weight w
// changes.  On the 128 x 64 x 15 grid those arrays take about 25 MB in total, less than
// the 152 x 228 KB of shared memory of a GB300.  So each tile loads its part once per month
// and every step then reads its matrices on chip; only the neighbours' state comes from L2.
// The state is kept interleaved, [cell][tracer], so one gather serves all tracers.
#pragma once

#include "tmm_kernels.cuh"

namespace m3d {

// Per-tile offsets into the global slice arrays (in doubles of one month).
struct ResidentTile {
    long long sp_base;     // first slot-lane of the tile's explicit slices
    int sp_n;              // slot-lanes of the tile (multiple of 32)
    int pad0;
    long long bk_base;     // first slot-lane of the tile's implicit slices
    int bk_n;
    int pad1;
};

struct ResidentParams {
    const ResidentTile *rt;
    int sp_max, bk_max;    // largest per-tile slot-lane counts (shared memory layout)
    // Tridiagonal form of the implicit matrices, when every monthly block is the inverse of
    // a tridiagonal matrix M = I - dt K (vertical diffusion): per month and cell the Thomas
    // factors of M, tri[m][f][cell] with f = 0: -l_k (sub-diagonal multiplier, 0 at the top),
    // 1: 1/d_k (inverse pivot), 2: -e_k / d_k (scaled super-diagonal, 0 at the bottom).
    const double *tri;
    long long tri_mstride; // 3 n
    const int *chains;     // per tile: chains (column, tracer, month) sorted by depth
    const int *chain_off;  // [ntiles+1]
};

// A chain packs: tile-local first cell of the column | layers << 16 | tracer << 23 | month << 27.
__host__ __device__ inline int pack_chain(int cb, int L, int t, int h) { return cb | (L << 16) | (t << 23) | (h << 27); }

// Shared memory layout of one tile, in bytes from the dynamic shared memory base.
struct ResidentLayout {
    int sa, sd, sb, sbd, si, tri, yt, z, ek, total;
};

__host__ __device__ inline ResidentLayout resident_layout(int ntr, int sp_max, int bk_max, int zmax, bool tri)
{
    ResidentLayout L;
    int o = 0;
    L.sa = o;  o += sp_max * 8;
    L.sd = o;  o += sp_max * 8;
    L.sb = o;  o += tri ? 0 : bk_max * 8;
    L.sbd = o; o += tri ? 0 : bk_max * 8;
    L.tri = o; o += tri ? 6 * zmax * 8 : 0;      // factors of months m0 and m1
    L.yt = o;  o += tri ? 2 * ntr * zmax * 8 : 0; // the two monthly solutions
    L.si = o;  o += sp_max * 4;
    o = (o + 15) & ~15;
    L.z = o;   o += ntr * zmax * 8;
    L.ek = o;  o += 2 * zmax * 8;
    L.total = (o + 15) & ~15;
    return L;
}

// Copy `count` doubles (a multiple of 32) from global to shared memory, 16 bytes per load.
__device__ __forceinline__ void copy_to_shared(double *dst, const double *__restrict__ src, int count)
{
    const double2 *s2 = reinterpret_cast<const double2 *>(src);
    double2 *d2 = reinterpret_cast<double2 *>(dst);
    for (int i = threadIdx.x; i < count / 2; i += blockDim.x) d2[i] = __ldg(s2 + i);
}

__device__ __forceinline__ void copy_to_shared_int(int *dst, const int *__restrict__ src, int count)
{
    const int4 *s4 = reinterpret_cast<const int4 *>(src);
    int4 *d4 = reinterpret_cast<int4 *>(dst);
    for (int i = threadIdx.x; i < count / 4; i += blockDim.x) d4[i] = __ldg(s4 + i);
}

// The explicit and implicit parts of one TMM step of one tile with its month resident in
// shared memory: z += A_exp(t_j) y_j (z holds the source increment already), then
// y_{j+1} = A_imp(t_j) z into the interleaved state.
template <int NTR, int MODEL, bool TRI>
__device__ __forceinline__ void transport_tile_resident(const StepParams &P, const Tile &T, int j,
                                                        const double *__restrict__ y, double *__restrict__ yn,
                                                        const double *sa, const double *sd, const double *sb,
                                                        const double *sbd, const int *si, double *z,
                                                        int sp_first, int bk_first)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int zmax = P.zmax;
    const double w = __ldg(P.wtab + j);
    const StateView<NTR, true, true> Y{y, P.n};

    // ---- explicit part from shared memory; neighbour state from L2
    const int *wl = P.sp_wlist + __ldg(P.sp_woff + blockIdx.x * (nwarps + 1) + warp);
    const int wn = __ldg(P.sp_woff + blockIdx.x * (nwarps + 1) + warp + 1) -
                   __ldg(P.sp_woff + blockIdx.x * (nwarps + 1) + warp);
    for (int ws = 0; ws < wn; ws++) {
        const int s = __ldg(wl + ws);
        const int len = __ldg(P.sp_len + s);
        const int base = (__ldg(P.sp_off + s) - sp_first) * 32 + lane;
        const int row = __ldg(P.sp_row + s * 32 + lane);
        double acc[NTR];
#pragma unroll
        for (int t = 0; t < NTR; t++) acc[t] = 0.0;
#pragma unroll 4
        for (int q = 0; q < len; q++) {
            const int idx = base + q * 32;
            double v[NTR];
            Y.gather(si[idx], v);
            const double a = fma(w, sd[idx], sa[idx]);
#pragma unroll
            for (int t = 0; t < NTR; t++) acc[t] = fma(a, v[t], acc[t]);
        }
        if (row >= 0) {
#pragma unroll
            for (int t = 0; t < NTR; t++)
                z[t * zmax + row] = ModelTraits<MODEL>::has_q ? acc[t] + z[t * zmax + row] : acc[t];
        }
    }
    __syncthreads();
    if (TRI) return;

    // ---- implicit part from shared memory into the interleaved y_{j+1}
    const int *bl = P.bk_wlist + __ldg(P.bk_woff + blockIdx.x * (nwarps + 1) + warp);
    const int bn = __ldg(P.bk_woff + blockIdx.x * (nwarps + 1) + warp + 1) -
                   __ldg(P.bk_woff + blockIdx.x * (nwarps + 1) + warp);
    for (int ws = 0; ws < bn; ws++) {
        const int s = __ldg(bl + ws);
        const int len = __ldg(P.bk_len + s);
        const int base = (__ldg(P.bk_off + s) - bk_first) * 32 + lane;
        const int row = __ldg(P.bk_row + s * 32 + lane);
        const int cb = __ldg(P.bk_cb + s * 32 + lane);
        const int Lc = __ldg(P.bk_L + s * 32 + lane);
        double acc[NTR];
#pragma unroll
        for (int t = 0; t < NTR; t++) acc[t] = 0.0;
#pragma unroll 4
        for (int c = 0; c < len; c++) {
            const int idx = base + c * 32;
            const double b = fma(w, sbd[idx], sb[idx]);
            const int zi = cb + (c < Lc ? c : 0);
#pragma unroll
            for (int t = 0; t < NTR; t++) acc[t] = fma(b, z[t * zmax + zi], acc[t]);
        }
        if (row >= 0) {
            double *o = yn + (size_t)(T.cell0 + row) * NTR;
            if (NTR % 2 == 0) {
#pragma unroll
                for (int t = 0; t < NTR; t += 2)
                    *reinterpret_cast<double2 *>(o + t) = make_double2(acc[t], acc[t + 1]);
            } else {
#pragma unroll
                for (int t = 0; t < NTR; t++) o[t] = acc[t];
            }
        }
    }
}

// Implicit part in tridiagonal form: y_{j+1} = z0 + w (z1 - z0) with z_h = M_{m_h}^{-1} z
// solved by Thomas' algorithm, one thread per (column, tracer, month) chain, then one
// combining pass.  Equal to (B_m0 + w (B_m1 - B_m0)) z up to rounding, because the monthly
// blocks are the inverses B_m = M_m^{-1}.
template <int NTR>
__device__ __forceinline__ void implicit_tridiagonal_tile(const StepParams &P, const ResidentParams &R,
                                                          const Tile &T, int j, const double *z,
                                                          const double *tl, double *yt, int ch0, int ch1,
                                                          double *__restrict__ yn)
{
    const int zmax = P.zmax;
    const double w = __ldg(P.wtab + j);
    for (int c = ch0 + (int)threadIdx.x; c < ch1; c += blockDim.x) {
        const int pc = __ldg(R.chains + c);
        const int cb = pc & 0xffff, L = (pc >> 16) & 0x7f, t = (pc >> 23) & 0xf, h = (pc >> 27) & 1;
        const double *nl = tl + (3 * h + 0) * zmax + cb;
        const double *rd = tl + (3 * h + 1) * zmax + cb;
        const double *ne = tl + (3 * h + 2) * zmax + cb;
        const double *zc = z + t * zmax + cb;
        double *x = yt + (h * NTR + t) * zmax + cb;
        // forward: x_k = z_k - l_k x_{k-1}, stored as x_k / d_k (off the dependency chain)
        double xk = zc[0];
        x[0] = xk * rd[0];
        for (int k = 1; k < L; k++) {
            xk = fma(nl[k], xk, zc[k]);
            x[k] = xk * rd[k];
        }
        // back: y_k = x_k / d_k - (e_k / d_k) y_{k+1}, one dependent FMA per layer
        double yk = x[L - 1];
        for (int k = L - 2; k >= 0; k--) {
            yk = fma(ne[k], yk, x[k]);
            x[k] = yk;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < T.ncell; i += blockDim.x) {
        double v[NTR];
#pragma unroll
        for (int t = 0; t < NTR; t++) {
            const double a = yt[t * zmax + i], b = yt[(NTR + t) * zmax + i];
            v[t] = fma(w, b - a, a);
        }
        double *o = yn + (size_t)(T.cell0 + i) * NTR;
        if (NTR % 2 == 0) {
#pragma unroll
            for (int t = 0; t < NTR; t += 2) *reinterpret_cast<double2 *>(o + t) = make_double2(v[t], v[t + 1]);
        } else {
#pragma unroll
            for (int t = 0; t < NTR; t++) o[t] = v[t];
        }
    }
}

template <int NTR, int MODEL, bool TRI>
__device__ __forceinline__ void year_resident(const StepParams &P, const ResidentParams &R, const SyncParams &S,
                                              double *buf0, double *buf1, int j0, int nsteps)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ int abort_flag;
    const int tile = blockIdx.x;
    const Tile T = P.tiles[tile];
    const ResidentTile RT = R.rt[tile];
    const ResidentLayout Ly = resident_layout(NTR, R.sp_max, R.bk_max, P.zmax, TRI);
    double *sa = reinterpret_cast<double *>(dsm + Ly.sa);
    double *sd = reinterpret_cast<double *>(dsm + Ly.sd);
    double *sb = reinterpret_cast<double *>(dsm + Ly.sb);
    double *sbd = reinterpret_cast<double *>(dsm + Ly.sbd);
    int *si = reinterpret_cast<int *>(dsm + Ly.si);
    double *z = reinterpret_cast<double *>(dsm + Ly.z);
    double *ek = reinterpret_cast<double *>(dsm + Ly.ek);
    double *tl = reinterpret_cast<double *>(dsm + Ly.tri);
    double *yt = reinterpret_cast<double *>(dsm + Ly.yt);
    const int ch0 = TRI ? __ldg(R.chain_off + tile) : 0, ch1 = TRI ? __ldg(R.chain_off + tile + 1) : 0;
    const int sp_first = T.sp0 < T.sp1 ? __ldg(P.sp_off + T.sp0) : 0;
    const int bk_first = T.bk0 < T.bk1 ? __ldg(P.bk_off + T.bk0) : 0;

    copy_to_shared_int(si, P.sp_col + RT.sp_base, RT.sp_n);
    int cur_month = -1;
    for (int s = 0; s < nsteps; s++) {
        const int j = (j0 + s) % P.nstep;
        const double *y = (s & 1) ? buf1 : buf0;
        double *yn = (s & 1) ? buf0 : buf1;
        const int m0 = __ldg(P.m0tab + j);
        if (m0 != cur_month) {
            // a new month: load this tile's matrices (independent of the state, so before the wait)
            copy_to_shared(sa, P.sp_a + (long long)m0 * P.sp_mstride + RT.sp_base, RT.sp_n);
            copy_to_shared(sd, P.sp_d + (long long)m0 * P.sp_mstride + RT.sp_base, RT.sp_n);
            if (TRI) {
                const int m1 = (m0 + 1) % P.nmonth;
                for (int h = 0; h < 2; h++)
                    for (int f = 0; f < 3; f++) {
                        const double *src = R.tri + (long long)(h ? m1 : m0) * R.tri_mstride + (long long)f * P.n + T.cell0;
                        double *dst = tl + (3 * h + f) * P.zmax;
                        for (int i = threadIdx.x; i < T.ncell; i += blockDim.x) dst[i] = __ldg(src + i);
                    }
            } else {
                copy_to_shared(sb, P.bk_b + (long long)m0 * P.bk_mstride + RT.bk_base, RT.bk_n);
                copy_to_shared(sbd, P.bk_d + (long long)m0 * P.bk_mstride + RT.bk_base, RT.bk_n);
            }
            cur_month = m0;
        }
        // The source term needs only this tile's own cells: the last warp waits for the
        // neighbouring tiles while the other warps compute it.
        const int nwork = blockDim.x - 32;
        if ((int)threadIdx.x < nwork) {
            if (ModelTraits<MODEL>::has_q) {
                const StateView<NTR, true, true> Y{y, P.n};
                ndop_source_tile<typename ModelTraits<MODEL>::scalar>(P, T, j, Y, z, ek, nwork, 1);
            }
        } else if (s > 0) {
            bool ok = wait_neighbours(S, tile, s, s);
            if (threadIdx.x == nwork) abort_flag = ok ? 0 : 1;
        }
        __syncthreads();
        if (s > 0 && abort_flag) return;
        transport_tile_resident<NTR, MODEL, TRI>(P, T, j, y, yn, sa, sd, sb, sbd, si, z, sp_first, bk_first);
        if (TRI) implicit_tridiagonal_tile<NTR>(P, R, T, j, z, tl, yt, ch0, ch1, yn);
        // the CTA barrier orders every thread's stores of y_{j+1} before thread 0's release
        __syncthreads();
        if (threadIdx.x == 0 && tile != S.withhold_tile) store_release(S.flags + tile, s + 1);
    }
}

// Layout conversions between the caller's [tracer][cell] and the interleaved [cell][tracer].
template <int NTR>
__global__ void k_interleave(int n, const double *__restrict__ src, double *__restrict__ dst)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int t = 0; t < NTR; t++) dst[(size_t)i * NTR + t] = src[(size_t)t * n + i];
}

template <int NTR>
__global__ void k_deinterleave(int n, const double *__restrict__ src, double *__restrict__ dst)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int t = 0; t < NTR; t++) dst[(size_t)t * n + i] = src[(size_t)i * NTR + t];
}

}  // namespace m3d
