// tmm_resident.cuh -- the year map (Metos3D, arXiv:1410.0204, Section 4) as one persistent
// launch whose tiles keep their month of transport matrices in shared memory, and the
// reverse (adjoint) sweep of the year map in the same form.
//
// Within one month of the year (240 of the 2880 steps) a tile reads the same arrays every
// step: A_m, A_{m+1} - A_m and the implicit operator of months m and m+1; only the
// interpolation weight w changes.  On the 128 x 64 x 15 grid those arrays take about 25 MB
// in total, less than the 152 x 228 KB of shared memory of a GB300.  So each tile loads its
// part once per month and every step then reads its matrices on chip; only the neighbours'
// state comes from L2.  The state is kept interleaved, [cell][tracer], so one gather
// serves all tracers.
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
    // 1: 1/d_k (inverse pivot), 2: -e_k / d_{k+1} (super-diagonal over the next pivot, 0 at the
    // bottom; the back substitution runs in u_k = d_k y_k).
    const double *tri;
    long long tri_mstride; // 3 n
    const int *chains;     // per tile: chains (column, tracer, month) sorted by depth
    const int *chain_off;  // [ntiles+1]
    // Per-step explicit operators, when the context keeps them: sp_b[j][slot-lane] =
    // A_m0(j) + w_j (A_m1(j) - A_m0(j)) in the slice layout of sp_a (sp_bstride slot-lanes per
    // step).  The year kernel then streams step j's values into shared memory instead of
    // interpolating every entry itself.  Null: interpolate in the kernel.
    const double *sp_b;
    long long sp_bstride;
};

// Thomas chains of at most this many layers run in registers (deeper ones through shared memory).
constexpr int kChainRegs = 16;

// A chain packs: tile-local first cell of the column | layers << 16 | tracer << 23 | month << 27.
__host__ __device__ inline int pack_chain(int cb, int L, int t, int h) { return cb | (L << 16) | (t << 23) | (h << 27); }

// ---- one-dimensional bulk copies (TMA) from global into shared memory, completed on an
// mbarrier.  Addresses and sizes are multiples of 16 bytes.
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make initialised barriers visible to the bulk-copy (async) proxy.
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Arrive on `bar` announcing `bytes` of transfer, then copy `bytes` from src (global) to dst
// (shared); the barrier's phase completes when the bytes have landed.  bytes == 0: a plain
// arrival.
__device__ __forceinline__ void bulk_copy_to_shared(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    if (bytes == 0) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_addr(bar)) : "memory");
        return;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_addr(dst)), "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Start bringing `bytes` at src (global) into L2; no completion to wait for.
__device__ __forceinline__ void prefetch_l2(const void *src, unsigned bytes)
{
    if (bytes) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(__cvta_generic_to_global(src)), "r"(bytes)
                            : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long *bar, unsigned parity)
{
    unsigned done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return done != 0;
}

// Wait until the phase of parity `parity` of `bar` has completed, at most timeout_ns.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity,
                                                  unsigned long long timeout_ns)
{
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_test(bar, parity))
        if (global_ns() - t0 > timeout_ns) return false;
    return true;
}

// Shared memory layout of one tile, in bytes from the dynamic shared memory base.
struct ResidentLayout {
    int sa, sd, sb, sbd, si, tri, yt, z, dq, ek, aux, total;
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
    L.dq = o;  o += ntr * zmax * 8;                  // source increment (written while z is)
    L.ek = o;  o += 2 * zmax * 8;
    L.aux = o; o += zmax * 8;
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

// Shared memory views of one tile.
struct TileSmem {
    double *sa, *sd, *sb, *sbd, *tl, *yt, *z, *dq, *ek, *aux;
    int *si;
    int sp_first, bk_first;     // first slot of the tile's explicit / implicit slices
};

__device__ __forceinline__ TileSmem tile_smem(unsigned char *dsm, const ResidentLayout &Ly, const StepParams &P,
                                              const Tile &T)
{
    TileSmem M;
    M.sa = reinterpret_cast<double *>(dsm + Ly.sa);
    M.sd = reinterpret_cast<double *>(dsm + Ly.sd);
    M.sb = reinterpret_cast<double *>(dsm + Ly.sb);
    M.sbd = reinterpret_cast<double *>(dsm + Ly.sbd);
    M.tl = reinterpret_cast<double *>(dsm + Ly.tri);
    M.yt = reinterpret_cast<double *>(dsm + Ly.yt);
    M.z = reinterpret_cast<double *>(dsm + Ly.z);
    M.dq = reinterpret_cast<double *>(dsm + Ly.dq);
    M.ek = reinterpret_cast<double *>(dsm + Ly.ek);
    M.aux = reinterpret_cast<double *>(dsm + Ly.aux);
    M.si = reinterpret_cast<int *>(dsm + Ly.si);
    M.sp_first = T.sp0 < T.sp1 ? __ldg(P.sp_off + T.sp0) : 0;
    M.bk_first = T.bk0 < T.bk1 ? __ldg(P.bk_off + T.bk0) : 0;
    return M;
}

// Load the explicit values of month m (A_m and A_{m+1} - A_m from the arrays a, d).
__device__ __forceinline__ void load_explicit_month(const StepParams &P, const ResidentTile &RT, const double *a,
                                                    const double *d, int m, const TileSmem &M)
{
    copy_to_shared(M.sa, a + (long long)m * P.sp_mstride + RT.sp_base, RT.sp_n);
    copy_to_shared(M.sd, d + (long long)m * P.sp_mstride + RT.sp_base, RT.sp_n);
}

// Load the implicit operator of months m and m+1: Thomas factors (TRI) or dense slices.
template <bool TRI>
__device__ __forceinline__ void load_implicit_month(const StepParams &P, const ResidentParams &R,
                                                    const ResidentTile &RT, const Tile &T, const double *tri,
                                                    const double *b, const double *bd, int m, const TileSmem &M)
{
    if (TRI) {
        const int m1 = (m + 1) % P.nmonth;
        for (int h = 0; h < 2; h++)
            for (int f = 0; f < 3; f++) {
                const double *src = tri + (long long)(h ? m1 : m) * R.tri_mstride + (long long)f * P.n + T.cell0;
                double *dst = M.tl + (3 * h + f) * P.zmax;
                for (int i = threadIdx.x; i < T.ncell; i += blockDim.x) dst[i] = __ldg(src + i);
            }
    } else {
        copy_to_shared(M.sb, b + (long long)m * P.bk_mstride + RT.bk_base, RT.bk_n);
        copy_to_shared(M.sbd, bd + (long long)m * P.bk_mstride + RT.bk_base, RT.bk_n);
    }
}

// Explicit part from shared memory: z[t][row] = (A_m0 + w D_m0) y for the tile's rows, plus
// z[t][row] when ADD (z then holds the source increment).  Neighbour state from L2.  Run by
// warp `warp` of `nwarps` warps that share the tile's slices as the deal (wlist, woff) gives.
// STEPOP: the step's interpolated values are already in shared memory at M.sa + sboff (same
// slice layout as sa; an offset from M.sa keeps the loads shared-memory loads).
template <int NTR, bool ADD, bool STEPOP = false>
__device__ __forceinline__ void spmv_resident(const StepParams &P, const Tile &T, double w,
                                              const double *__restrict__ y, const TileSmem &M,
                                              const int *wlist, const int *woff, int nwarps, int warp,
                                              int sboff = 0)
{
    const int lane = threadIdx.x & 31;
    const int zmax = P.zmax;
    const StateView<NTR, true, true> Y{y, P.n};
    const int *wl = wlist + __ldg(woff + blockIdx.x * (nwarps + 1) + warp);
    const int wn = __ldg(woff + blockIdx.x * (nwarps + 1) + warp + 1) - __ldg(woff + blockIdx.x * (nwarps + 1) + warp);
    for (int ws = 0; ws < wn; ws++) {
        const int s = __ldg(wl + ws);
        const int len = __ldg(P.sp_len + s);
        const int base = (__ldg(P.sp_off + s) - M.sp_first) * 32 + lane;
        const int row = __ldg(P.sp_row + s * 32 + lane);
        double acc[NTR];
#pragma unroll
        for (int t = 0; t < NTR; t++) acc[t] = 0.0;
#pragma unroll 4
        for (int q = 0; q < len; q++) {
            const int idx = base + q * 32;
            double v[NTR];
            Y.gather(M.si[idx], v);
            const double a = STEPOP ? M.sa[sboff + idx] : fma(w, M.sd[idx], M.sa[idx]);
#pragma unroll
            for (int t = 0; t < NTR; t++) acc[t] = fma(a, v[t], acc[t]);
        }
        if (row >= 0) {
#pragma unroll
            for (int t = 0; t < NTR; t++) M.z[t * zmax + row] = ADD ? acc[t] + M.z[t * zmax + row] : acc[t];
        }
    }
}

// The explicit part by all warps of the CTA.
template <int NTR, bool ADD>
__device__ __forceinline__ void spmv_resident(const StepParams &P, const Tile &T, double w,
                                              const double *__restrict__ y, const TileSmem &M)
{
    spmv_resident<NTR, ADD>(P, T, w, y, M, P.sp_wlist, P.sp_woff, (int)(blockDim.x >> 5), (int)(threadIdx.x >> 5));
}

// Write the tile's values v[t] of one cell into the interleaved state.
template <int NTR>
__device__ __forceinline__ void store_cell(double *__restrict__ yn, int cell, const double *v)
{
    double *o = yn + (size_t)cell * NTR;
    if (NTR % 2 == 0) {
#pragma unroll
        for (int t = 0; t < NTR; t += 2) *reinterpret_cast<double2 *>(o + t) = make_double2(v[t], v[t + 1]);
    } else {
#pragma unroll
        for (int t = 0; t < NTR; t++) o[t] = v[t];
    }
}

// Implicit part, dense blocks from shared memory: yn = (B_m0 + w (B_m1 - B_m0)) z.
template <int NTR>
__device__ __forceinline__ void implicit_dense_resident(const StepParams &P, const Tile &T, double w,
                                                        const TileSmem &M, double *__restrict__ yn)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int zmax = P.zmax;
    const int *bl = P.bk_wlist + __ldg(P.bk_woff + blockIdx.x * (nwarps + 1) + warp);
    const int bn = __ldg(P.bk_woff + blockIdx.x * (nwarps + 1) + warp + 1) -
                   __ldg(P.bk_woff + blockIdx.x * (nwarps + 1) + warp);
    for (int ws = 0; ws < bn; ws++) {
        const int s = __ldg(bl + ws);
        const int len = __ldg(P.bk_len + s);
        const int base = (__ldg(P.bk_off + s) - M.bk_first) * 32 + lane;
        const int row = __ldg(P.bk_row + s * 32 + lane);
        const int cb = __ldg(P.bk_cb + s * 32 + lane);
        const int Lc = __ldg(P.bk_L + s * 32 + lane);
        double acc[NTR];
#pragma unroll
        for (int t = 0; t < NTR; t++) acc[t] = 0.0;
#pragma unroll 4
        for (int c = 0; c < len; c++) {
            const int idx = base + c * 32;
            const double b = fma(w, M.sbd[idx], M.sb[idx]);
            const int zi = cb + (c < Lc ? c : 0);
#pragma unroll
            for (int t = 0; t < NTR; t++) acc[t] = fma(b, M.z[t * zmax + zi], acc[t]);
        }
        if (row >= 0) store_cell<NTR>(yn, T.cell0 + row, acc);
    }
}

// Implicit part in tridiagonal form: yn = (1 - w) M0^{-1} z + w M1^{-1} z, each solve by
// Thomas' algorithm, one thread per (column, tracer, month) chain.  The chains back-substitute
// the unknowns u_k = d_k y_k with the factors (-l_k, 1/d_k, -e_k/d_{k+1}) -- two multiply-adds
// per layer, the serial part of the phase -- while the threads without a chain form the blend
// weights (1 - w)/d_k and w/d_k of every cell; one combining pass then writes
// (1 - w)/d0_k u0_k + w/d1_k u1_k.  Equal to (B_m0 + w (B_m1 - B_m0)) z up to rounding,
// because the monthly blocks are the inverses B_m = M_m^{-1}.
// The tile's chain range and this thread's first chain descriptor: the same every step, so a
// sweep loads them once (their loads would otherwise start every step's Thomas phase).
struct ChainPre {
    int ch0, ch1, pc0;
};

__device__ __forceinline__ ChainPre chain_pre(const ResidentParams &R)
{
    ChainPre C;
    C.ch0 = __ldg(R.chain_off + blockIdx.x);
    C.ch1 = __ldg(R.chain_off + blockIdx.x + 1);
    const int c = C.ch0 + (int)threadIdx.x;
    C.pc0 = c < C.ch1 ? __ldg(R.chains + c) : 0;
    return C;
}

template <int NTR, bool ADD_DQ>
__device__ __forceinline__ void implicit_tri_resident(const StepParams &P, const ResidentParams &R, const Tile &T,
                                                      double w, const TileSmem &M, double *__restrict__ yn,
                                                      const ChainPre &CP)
{
    const int zmax = P.zmax;
    const int ch0 = CP.ch0, ch1 = CP.ch1;
    const int nthreads = (int)blockDim.x, tid = (int)threadIdx.x;
    const int chain_threads = min(nthreads, ((ch1 - ch0 + 31) / 32) * 32);
    double *c0 = M.ek, *c1 = M.ek + zmax;     // blend weights (the source term's scratch is free now)
    if (tid < chain_threads) {
        for (int c = ch0 + tid; c < ch1; c += chain_threads) {
            const int pc = c == ch0 + tid ? CP.pc0 : __ldg(R.chains + c);
            const int cb = pc & 0xffff, L = (pc >> 16) & 0x7f, t = (pc >> 23) & 0xf, h = (pc >> 27) & 1;
            const double *nl = M.tl + (3 * h + 0) * zmax + cb;
            const double *ne = M.tl + (3 * h + 2) * zmax + cb;
            const double *zc = M.z + t * zmax + cb;
            const double *dqc = M.dq + t * zmax + cb;
            double *x = M.yt + (h * NTR + t) * zmax + cb;
            // the right-hand side A_exp y_j + dt q(y_j): the explicit part and the source term's
            // increment, added here (off the chain's dependency) rather than in a pass of their own
            auto rhs = [&](int k) { return ADD_DQ ? zc[k] + dqc[k] : zc[k]; };
            if (L <= kChainRegs) {
                // the chain in registers, unrolled: every factor and right-hand side is loaded
                // ahead of the dependent multiply-adds, which then run back to back
                double gk[kChainRegs];
                double g = 0.0;
#pragma unroll
                for (int k = 0; k < kChainRegs; k++)
                    if (k < L) {
                        g = fma(nl[k], g, rhs(k));
                        gk[k] = g;
                    }
                double u = 0.0;
#pragma unroll
                for (int k = kChainRegs - 1; k >= 0; k--)
                    if (k < L) {
                        u = fma(ne[k], u, gk[k]);
                        x[k] = u;
                    }
                continue;
            }
            // forward: g_k = z_k - l_k g_{k-1} (l_0 = 0)
            double g = 0.0;
            for (int k = 0; k < L; k++) {
                g = fma(nl[k], g, rhs(k));
                x[k] = g;
            }
            // back: u_k = g_k - (e_k / d_{k+1}) u_{k+1} (nothing below the bottom layer)
            double u = 0.0;
            for (int k = L - 1; k >= 0; k--) {
                u = fma(ne[k], u, x[k]);
                x[k] = u;
            }
        }
    }
    if (tid >= chain_threads || chain_threads == nthreads) {
        const int t0 = chain_threads == nthreads ? 0 : chain_threads;
        for (int i = tid - t0; i < T.ncell; i += nthreads - t0) {
            c0[i] = (1.0 - w) * M.tl[1 * zmax + i];
            c1[i] = w * M.tl[4 * zmax + i];
        }
    }
    __syncthreads();
    for (int i = tid; i < T.ncell; i += nthreads) {
        double v[NTR];
        const double a = c0[i], b = c1[i];
#pragma unroll
        for (int t = 0; t < NTR; t++) v[t] = fma(a, M.yt[t * zmax + i], b * M.yt[(NTR + t) * zmax + i]);
        store_cell<NTR>(yn, T.cell0 + i, v);
    }
}

template <int NTR, bool TRI, bool ADD_DQ = false>
__device__ __forceinline__ void implicit_resident(const StepParams &P, const ResidentParams &R, const Tile &T,
                                                  double w, const TileSmem &M, double *__restrict__ yn,
                                                  const ChainPre *CP = nullptr)
{
    if (TRI) {
        if (CP) implicit_tri_resident<NTR, ADD_DQ>(P, R, T, w, M, yn, *CP);
        else implicit_tri_resident<NTR, ADD_DQ>(P, R, T, w, M, yn, chain_pre(R));
    } else {
        if (ADD_DQ) {           // the dense form reads z once per block entry: add the increment first
            const int nc = T.ncell, zmax = P.zmax;
            for (int e = threadIdx.x; e < NTR * nc; e += blockDim.x) {
                const int t = e / nc, i = e - t * nc;
                M.z[t * zmax + i] += M.dq[t * zmax + i];
            }
            __syncthreads();
        }
        implicit_dense_resident<NTR>(P, T, w, M, yn);
    }
}

constexpr int kWarpsPerTile = kThreads / 32;   // releases per tile and step of the resident year kernel

// The year (or nsteps steps from step j0) with the tiles' months resident in shared memory.
// State of step s (interleaved): base + (s mod period) * stride; period 2 is a ping-pong,
// period nsteps + 1 keeps every state (the trajectory an adjoint sweep reads back).
//
// With per-step explicit operators (R.sp_b) the two explicit arrays of shared memory become a
// double buffer: step s reads buffer s mod 2, and once every thread is past step s's explicit
// part a bulk copy brings step s+1's values into the other buffer (last read in step s-1)
// while the tile solves the implicit part.  The copy reads from L2: step s+2's values are
// prefetched from HBM into L2 at the same time, a step ahead of their copy, which keeps
// HBM latency out of the step.  Every wait is bounded; a tile that gives up lets its copy in
// flight land before it returns.
template <int NTR, int MODEL, bool TRI>
__device__ __forceinline__ void year_resident(const StepParams &P, const ResidentParams &R, const SyncParams &S,
                                              double *base, long long stride, int period, int j0, int nsteps)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ int abort_flag;
    __shared__ __align__(8) unsigned long long opbar[2];
    const int tile = blockIdx.x;
    const Tile T = P.tiles[tile];
    const ResidentTile RT = R.rt[tile];
    const ResidentLayout Ly = resident_layout(NTR, R.sp_max, R.bk_max, P.zmax, TRI);
    const TileSmem M = tile_smem(dsm, Ly, P, T);
    // buffers: M.sa and M.sd = M.sa + R.sp_max (no copy is started for an empty launch)
    const bool stepop = R.sp_b != nullptr && nsteps > 0;
    const unsigned opbytes = (unsigned)RT.sp_n * 8u;
    const int copier = kThreads - 32;          // a thread off the implicit part's critical path
    auto op_src = [&](int s) { return R.sp_b + (long long)((j0 + s) % P.nstep) * R.sp_bstride + RT.sp_base; };
    auto fetch_operator = [&](int s) {         // step s's values into buffer s mod 2; s+1's into L2
        bulk_copy_to_shared((s & 1) ? M.sd : M.sa, op_src(s), opbytes, &opbar[s & 1]);
        if (s + 1 < nsteps) prefetch_l2(op_src(s + 1), opbytes);
    };

    if (stepop && threadIdx.x == 0) {
        mbar_init(&opbar[0], 1);
        mbar_init(&opbar[1], 1);
        mbar_init_fence();
        fetch_operator(0);
    }
    copy_to_shared_int(M.si, P.sp_col + RT.sp_base, RT.sp_n);
    ChainPre CP{0, 0, 0};
    if (TRI) CP = chain_pre(R);
    __syncthreads();
    int cur_month = -1;
    for (int s = 0; s < nsteps; s++) {
        const int j = (j0 + s) % P.nstep;
        const double *y = base + (long long)(s % period) * stride;
        double *yn = base + (long long)((s + 1) % period) * stride;
        const int m0 = __ldg(P.m0tab + j);
        const double w = __ldg(P.wtab + j);
        if (m0 != cur_month) {
            // a new month: load this tile's matrices (independent of the state, so before the wait)
            if (!stepop) load_explicit_month(P, RT, P.sp_a, P.sp_d, m0, M);
            load_implicit_month<TRI>(P, R, RT, T, R.tri, P.bk_b, P.bk_d, m0, M);
            cur_month = m0;
            __syncthreads();
        }
        // Two groups work at once.  The source term needs only this tile's own cells, so the
        // last kQWarps warps compute it into dq straight away; the explicit group waits for
        // the neighbouring tiles (warp 0 polls, the others at a named barrier) and then
        // forms z = A_exp y.  The source term's divisions and sums are latency-bound and the
        // explicit part is FP64-throughput-bound, so together they keep the FP64 pipes busier.
        if ((int)threadIdx.x >= kSpThreads) {
            if (MODEL == kModelNdopLinear) {
                const StateView<NTR, true, true> Y{y, P.n};
                ndop_source_tile_linear(P, T, j, Y, M.dq, M.ek, kQThreads, 2, kSpThreads);
            } else if (ModelTraits<MODEL>::has_q) {
                const StateView<NTR, true, true> Y{y, P.n};
                ndop_source_tile<typename ModelTraits<MODEL>::scalar>(P, T, j, Y, M.dq, M.ek, kQThreads, 2,
                                                                      kSpThreads);
            }
        } else {
            if (s > 0 || stepop) {
                if (threadIdx.x < 32) {
                    bool ok = s > 0 ? wait_neighbours(S, tile, kWarpsPerTile * s, s) : true;
                    if (ok && stepop && !mbar_wait_bounded(&opbar[s & 1], (s >> 1) & 1, S.timeout_ns)) {
                        if (atomicCAS(S.status, 0, 1) == 0) {
                            S.status[1] = tile;
                            S.status[2] = s;
                        }
                        ok = false;
                    }
                    ok = __all_sync(0xffffffffu, ok);
                    if (threadIdx.x == 0) abort_flag = ok ? 0 : 1;
                }
                barrier_sub(3);
            }
            if (stepop) {
                // every reader observes the completed copy itself (it has, so this returns at once)
                if (!abort_flag) {
                    if (mbar_wait_bounded(&opbar[s & 1], (s >> 1) & 1, S.timeout_ns))
                        spmv_resident<NTR, false, true>(P, T, w, y, M, P.sp_wlist_g, P.sp_woff_g, kSpThreads / 32,
                                                        (int)(threadIdx.x >> 5), (s & 1) * R.sp_max);
                    else if (atomicCAS(S.status, 0, 1) == 0) {
                        S.status[1] = tile;
                        S.status[2] = s;
                    }
                }
            } else if (s == 0 || !abort_flag) {
                spmv_resident<NTR, false>(P, T, w, y, M, P.sp_wlist_g, P.sp_woff_g, kSpThreads / 32,
                                          (int)(threadIdx.x >> 5));
            }
        }
        __syncthreads();
        if ((s > 0 || stepop) && abort_flag) {
            // The copy of step s may still be in flight (no later one was issued); it depends on
            // no other tile, so it lands within the bound unless the GPU is failing.  If the
            // bound runs out anyway, status[3] records it before the CTA retires.
            if (stepop && threadIdx.x == 0 && !mbar_wait_bounded(&opbar[s & 1], (s >> 1) & 1, S.timeout_ns))
                atomicExch(S.status + 3, 1);
            return;
        }
        if (stepop && threadIdx.x == copier && s + 1 < nsteps) fetch_operator(s + 1);
        implicit_resident<NTR, TRI, ModelTraits<MODEL>::has_q>(P, R, T, w, M, yn, &CP);
        // Every warp publishes its own stores of y_{j+1} as soon as they are made: the tile's
        // counter gains one per warp, and the neighbours wait for kWarpsPerTile (s + 1).  No
        // CTA barrier stands before the release, and each warp's fence waits only for its own
        // stores.  The barrier after it keeps the tile's own next step behind all of them.
        __syncwarp();
        if ((threadIdx.x & 31) == 0 && tile != S.withhold_tile) add_release(S.flags + tile, 1);
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// Reverse (adjoint) sweep.  For one step y_{j+1} = B_j (A_j y_j + dq_j(y_j, u)) and the
// cotangent zbar_j = B_j^T ybar_{j+1}:
//     ybar_j = A_j^T zbar_j + (d dq_j / dy)^T zbar_j,   ubar += (d dq_j / du)^T zbar_j,
// then zbar_{j-1} = B_{j-1}^T ybar_j.  The transposed operators have the same slice layouts
// as the forward ones (the explicit pattern is structurally symmetric), so the same
// device code applies them.

// Per-call tables and outputs of the adjoint of the PO4-DOP term.
struct AdjointParams {
    const double *mfrac_b;     // [n] d mfrac / d b (aphotic cells)
    const double *zc;          // [n] layer-centre depth
    const int *col_list;       // per tile: its columns, tile-local first cell | layers << 16
    const int *col_off;        // [ntiles+1]
    double *ubar_part;         // [ntiles][8] parameter gradient of each tile
};

// Reverse of the PO4-DOP increment dq = ds q(y) (one internal step) on the tile's cells:
// given zbar (cotangent of dq, global interleaved) and y_j, add (d dq/dy)^T zbar into M.z
// (the tile's ybar_j) and (d dq/du)^T zbar into ub[7].
//   euphotic: f = alpha' N/(N+K_N) I/(I+K_I), qN = -f + lambda D, qD = sigma f - lambda D
//   E = (1 - sigma) sum f h;  aphotic: qN = E mfrac + lambda D, qD = -lambda D
//   shallow column: the bottom layer also gets E / h.
template <int NTR>
__device__ __forceinline__ void ndop_source_adjoint_tile(const StepParams &P, const AdjointParams &A, const Tile &T,
                                                         int j, const double *__restrict__ y,
                                                         const double *__restrict__ zbar, const TileSmem &M,
                                                         double *ub)
{
    const int zmax = P.zmax;
    const double alpha = __ldg(P.qpar + kQAlpha), sigma = __ldg(P.qpar + kQSigma);
    const double lambda = __ldg(P.qpar + kQLambda), KN = __ldg(P.qpar + kQKN);
    const double KI = __ldg(P.qpar + kQKI), oms = __ldg(P.qpar + kQOneMinusSigma);
    const double ds = P.ds;
    const double *I0row = P.I0tab + (size_t)j * P.nulat;
    double *fk = M.ek;                 // [zmax] production f of euphotic cells
    double *ehk = M.ek + zmax;         // [zmax] (1 - sigma) f h of euphotic cells
    double *Ebar = M.aux;              // per column, at its first cell
    // (a) forward production of the euphotic cells
    for (int e = T.eu0 + (int)threadIdx.x; e < T.eu1; e += blockDim.x) {
        const int i = __ldg(P.eu_list + e);
        const int cell = T.cell0 + i;
        const double I = __ldg(I0row + __ldg(P.cell_ulat + cell)) * __ldg(P.atten + cell);
        const double N = __ldcg(y + (size_t)cell * NTR);
        const double f = (alpha * N * I) / ((N + KN) * (I + KI));
        fk[i] = f;
        ehk[i] = oms * f * __ldg(P.h + cell);
    }
    __syncthreads();
    // (b) per column: the cotangent of its export, and the Martin exponent's gradient
    const int c0 = __ldg(A.col_off + blockIdx.x), c1 = __ldg(A.col_off + blockIdx.x + 1);
    for (int c = c0 + (int)threadIdx.x; c < c1; c += blockDim.x) {
        const int pc = __ldg(A.col_list + c);
        const int cb = pc & 0xffff, L = pc >> 16;
        const int neu = L < kEuphotic ? L : kEuphotic;
        double E = 0.0, sfh = 0.0;
        for (int k = 0; k < neu; k++) {
            E += ehk[cb + k];
            sfh += fk[cb + k] * __ldg(P.h + T.cell0 + cb + k);
        }
        double eb = 0.0, bb = 0.0;
        for (int k = neu; k < L; k++) {
            const int cell = T.cell0 + cb + k;
            const double qbN = ds * __ldcg(zbar + (size_t)cell * NTR);
            eb = fma(qbN, __ldg(P.mfrac + cell), eb);
            bb = fma(qbN * E, __ldg(A.mfrac_b + cell), bb);
        }
        if (L <= kEuphotic) {
            const int cell = T.cell0 + cb + L - 1;
            eb += ds * __ldcg(zbar + (size_t)cell * NTR) / __ldg(P.h + cell);
        }
        Ebar[cb] = eb;
        ub[6] += bb;
        ub[2] -= eb * sfh;                        // d E / d sigma = -sum f h
    }
    __syncthreads();
    // (c) every cell: DOP remineralisation; euphotic cells: production
    for (int i = threadIdx.x; i < T.ncell; i += blockDim.x) {
        const int cell = T.cell0 + i;
        const int k = __ldg(P.cell_kl + cell) & 0xff;
        const double qbN = ds * __ldcg(zbar + (size_t)cell * NTR);
        const double qbD = ds * __ldcg(zbar + (size_t)cell * NTR + 1);
        const double D = __ldcg(y + (size_t)cell * NTR + 1);
        const double dl = qbN - qbD;
        M.z[zmax + i] += lambda * dl;            // d q / d DOP
        ub[3] += dl * D;                          // d q / d lambda
        if (k < kEuphotic) {
            const double N = __ldcg(y + (size_t)cell * NTR);
            const double I = __ldg(I0row + __ldg(P.cell_ulat + cell)) * __ldg(P.atten + cell);
            const double f = fk[i];
            const double fb = Ebar[i - k] * oms * __ldg(P.h + cell) - qbN + sigma * qbD;
            ub[2] += qbD * f;
            const double NK = N + KN, IK = I + KI;
            const double Mm = N / NK, LF = I / IK;
            M.z[i] += fb * alpha * LF * (KN / (NK * NK));            // d f / d N
            ub[1] += fb * 360.0 * Mm * LF;                            // d f / d alpha (alpha per day)
            ub[4] += fb * alpha * LF * (-N / (NK * NK));              // d f / d K_N
            ub[5] += fb * alpha * Mm * (-I / (IK * IK));              // d f / d K_I
            ub[0] += fb * alpha * Mm * (KI / (IK * IK)) * (-__ldg(A.zc + cell) * I);   // d f / d k_w
        }
    }
}

// Reverse sweep over steps j0 + nsteps - 1 down to j0.  traj: the interleaved forward
// states y_{j0} .. y_{j0+nsteps-1} (stride apart); ybar_in: cotangent of y_{j0+nsteps}; out:
// cotangent of y_{j0}.  zb0, zb1: the interleaved ping-pong of zbar.  PT and RTp carry the
// transposed operators (same layouts as the forward ones).
template <int NTR, bool TRI, bool STREAM = false>
__device__ __forceinline__ void year_adjoint_resident(const StepParams &PT, const ResidentParams &RTp,
                                                      const SyncParams &S, const AdjointParams &A,
                                                      const double *traj, long long stride,
                                                      const double *ybar_in, double *out, double *zb0, double *zb1,
                                                      int j0, int nsteps)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ int abort_flag;
    __shared__ double red[kThreads / 32][7];
    __shared__ __align__(8) unsigned long long opbar[2];
    const int tile = blockIdx.x;
    const Tile T = PT.tiles[tile];
    const ResidentTile RT = RTp.rt[tile];
    const int zmax = PT.zmax;
    // STREAM: the operators are read from global memory where they lie (the month's slices of
    // the tile), only the tile's cotangent and the source term's scratch sit in shared memory,
    // and the implicit part uses the dense form (TRI must be false)
    static_assert(!(STREAM && TRI), "the streaming sweep applies dense implicit blocks");
    TileSmem M;
    if (STREAM) {
        double *base = reinterpret_cast<double *>(dsm);
        M.z = base;
        M.ek = base + NTR * zmax;
        M.aux = M.ek + 2 * zmax;
        M.dq = M.tl = M.yt = nullptr;
        M.sa = M.sd = M.sb = M.sbd = nullptr;
        M.si = const_cast<int *>(PT.sp_col) + RT.sp_base;
        M.sp_first = T.sp0 < T.sp1 ? __ldg(PT.sp_off + T.sp0) : 0;
        M.bk_first = T.bk0 < T.bk1 ? __ldg(PT.bk_off + T.bk0) : 0;
    } else {
        const ResidentLayout Ly = resident_layout(NTR, RTp.sp_max, RTp.bk_max, PT.zmax, TRI);
        M = tile_smem(dsm, Ly, PT, T);
        copy_to_shared_int(M.si, PT.sp_col + RT.sp_base, RT.sp_n);
    }
    double ub[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    // the month's operators: staged in shared memory, or pointed at where they lie
    auto explicit_month = [&](int m) {
        if (STREAM) {
            M.sa = const_cast<double *>(PT.sp_a) + (long long)m * PT.sp_mstride + RT.sp_base;
            M.sd = const_cast<double *>(PT.sp_d) + (long long)m * PT.sp_mstride + RT.sp_base;
        } else {
            load_explicit_month(PT, RT, PT.sp_a, PT.sp_d, m, M);
        }
    };
    auto implicit_month = [&](int m) {
        if (STREAM) {
            M.sb = const_cast<double *>(PT.bk_b) + (long long)m * PT.bk_mstride + RT.bk_base;
            M.sbd = const_cast<double *>(PT.bk_d) + (long long)m * PT.bk_mstride + RT.bk_base;
        } else {
            load_implicit_month<TRI>(PT, RTp, RT, T, RTp.tri, PT.bk_b, PT.bk_d, m, M);
        }
    };
    int exp_month = -1, imp_month = -1;
    // With per-step transposed operators (RTp.sp_b): the explicit arrays become a double
    // buffer, step s (j = j0 + nsteps - 1 - s) reads buffer s mod 2, and once every thread is
    // past step s's explicit part a bulk copy brings step s+1's values into the other buffer,
    // step s+2's being prefetched into L2 meanwhile (as in the forward sweep).
    const bool stepop = !STREAM && RTp.sp_b != nullptr && nsteps > 0;
    const unsigned opbytes = (unsigned)RT.sp_n * 8u;
    auto op_src = [&](int s) {
        return RTp.sp_b + (long long)((j0 + nsteps - 1 - s) % PT.nstep) * RTp.sp_bstride + RT.sp_base;
    };
    auto fetch_operator = [&](int s) {
        bulk_copy_to_shared((s & 1) ? M.sd : M.sa, op_src(s), opbytes, &opbar[s & 1]);
        if (s + 1 < nsteps) prefetch_l2(op_src(s + 1), opbytes);
    };
    if (stepop && threadIdx.x == 0) {
        mbar_init(&opbar[0], 1);
        mbar_init(&opbar[1], 1);
        mbar_init_fence();
        fetch_operator(0);
    }
    // zbar_{last} = B_last^T ybar_in on the tile's own cells
    {
        const int j = (j0 + nsteps - 1) % PT.nstep;
        const int m = __ldg(PT.m0tab + j);
        implicit_month(m);
        imp_month = m;
        for (int i = threadIdx.x; i < T.ncell; i += blockDim.x)
            for (int t = 0; t < NTR; t++) M.z[t * zmax + i] = __ldcg(ybar_in + (size_t)(T.cell0 + i) * NTR + t);
        __syncthreads();
        implicit_resident<NTR, TRI>(PT, RTp, T, __ldg(PT.wtab + j), M, zb0);
        __syncthreads();
        if (threadIdx.x == 0 && tile != S.withhold_tile) store_release(S.flags + tile, 1);
    }
    bool aborted = false;
    for (int s = 0; s < nsteps; s++) {
        const int j = (j0 + nsteps - 1 - s) % PT.nstep;
        const double *zb = (s & 1) ? zb1 : zb0;
        double *zn = (s & 1) ? zb0 : zb1;
        const double *y = traj + (long long)(nsteps - 1 - s) * stride;
        const int m = __ldg(PT.m0tab + j);
        if (!stepop && m != exp_month) {
            explicit_month(m);
            exp_month = m;
        }
        if (threadIdx.x < 32) {
            bool ok = wait_neighbours(S, tile, s + 1, s);
            if (threadIdx.x == 0) abort_flag = ok ? 0 : 1;
        }
        __syncthreads();
        if (abort_flag) {
            // step s's copy may be in flight; it depends on no other tile (status[3] if the bound
            // runs out anyway)
            if (stepop && threadIdx.x == 0 && !mbar_wait_bounded(&opbar[s & 1], (s >> 1) & 1, S.timeout_ns))
                atomicExch(S.status + 3, 1);
            aborted = true;
            break;
        }
        if (stepop) {
            // every reader observes the completed copy itself
            if (mbar_wait_bounded(&opbar[s & 1], (s >> 1) & 1, S.timeout_ns)) {
                spmv_resident<NTR, false, true>(PT, T, 0.0, zb, M, PT.sp_wlist, PT.sp_woff, (int)(blockDim.x >> 5),
                                                (int)(threadIdx.x >> 5), (s & 1) * RTp.sp_max);   // A_j^T zbar_j
            } else {
                if (atomicCAS(S.status, 0, 1) == 0) {
                    S.status[1] = tile;
                    S.status[2] = s;
                }
                abort_flag = 1;
            }
            __syncthreads();
            if (abort_flag) {
                if (threadIdx.x == 0 && !mbar_wait_bounded(&opbar[s & 1], (s >> 1) & 1, S.timeout_ns))
                    atomicExch(S.status + 3, 1);
                aborted = true;
                break;
            }
            if (threadIdx.x == kThreads - 32 && s + 1 < nsteps) fetch_operator(s + 1);
        } else {
            spmv_resident<NTR, false>(PT, T, __ldg(PT.wtab + j), zb, M);   // ybar_j = A_j^T zbar_j
            __syncthreads();
        }
        ndop_source_adjoint_tile<NTR>(PT, A, T, j, y, zb, M, ub);           // + (d dq/dy)^T zbar_j
        __syncthreads();
        if (s + 1 < nsteps) {
            const int jm = (j + PT.nstep - 1) % PT.nstep;
            const int mm = __ldg(PT.m0tab + jm);
            if (mm != imp_month) {
                implicit_month(mm);
                imp_month = mm;
                __syncthreads();
            }
            implicit_resident<NTR, TRI>(PT, RTp, T, __ldg(PT.wtab + jm), M, zn);   // zbar_{j-1}
        } else {
            for (int i = threadIdx.x; i < T.ncell; i += blockDim.x) {
                double v[NTR];
                for (int t = 0; t < NTR; t++) v[t] = M.z[t * zmax + i];
                store_cell<NTR>(out, T.cell0 + i, v);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && tile != S.withhold_tile) store_release(S.flags + tile, s + 2);
    }
    if (aborted) return;
    // the tile's parameter gradient: fixed-order block reduction
    for (int k = 0; k < 7; k++) {
        double v = ub[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) v += red[w][threadIdx.x];
        A.ubar_part[(size_t)tile * 8 + threadIdx.x] = v;
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
