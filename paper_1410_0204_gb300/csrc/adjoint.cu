// adjoint.cu -- the reverse (adjoint) year map and the gradient with respect to the model
// parameters (Metos3D, arXiv:1410.0204: parameter optimisation, Sections 1 and 9; exact
// derivatives by algorithmic differentiation, Section 6).
//
// For y1 = phi(y0; u) and a cotangent ybar1 the library returns ybar0 = phi_y^T ybar1 and
// ubar = phi_u^T ybar1.  The states of the year are needed in reverse order: the forward
// sweep keeps one checkpoint every K steps, and each segment is recomputed (all its states
// kept) just before its reverse sweep, so the cost is about two forward years and one
// reverse year, and the memory about K states.
#include <cmath>
#include <cstring>
#include <vector>

#include "adjoint.h"

namespace {

template <bool TRI>
__global__ void __launch_bounds__(m3d::kThreads, 1) k_year_adjoint(StepParams PT, m3d::ResidentParams RT,
                                                                m3d::SyncParams S, m3d::AdjointParams A,
                                                                const double *traj, long long stride,
                                                                const double *ybar_in, double *out, double *zb0,
                                                                double *zb1, int j0, int nsteps)
{
    m3d::year_adjoint_resident<2, TRI>(PT, RT, S, A, traj, stride, ybar_in, out, zb0, zb1, j0, nsteps);
}

// The same sweep reading the operators from global memory (grids whose tiles' months do not
// fit in shared memory).
__global__ void __launch_bounds__(m3d::kThreads, 1) k_year_adjoint_stream(StepParams PT, m3d::ResidentParams RT,
                                                                       m3d::SyncParams S, m3d::AdjointParams A,
                                                                       const double *traj, long long stride,
                                                                       const double *ybar_in, double *out,
                                                                       double *zb0, double *zb1, int j0, int nsteps)
{
    m3d::year_adjoint_resident<2, false, true>(PT, RT, S, A, traj, stride, ybar_in, out, zb0, zb1, j0, nsteps);
}

// d mfrac / d b on aphotic cells (the parameter gradient of the Martin profile).
__global__ void k_martin_b(int n, const int *cell_kl, const double *h, const double *u, double *mfrac_b)
{
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= n) return;
    int kl = cell_kl[cell];
    int k = kl & 0xff, L = kl >> 8;
    if (L <= m3d::kEuphotic || k < m3d::kEuphotic) { mfrac_b[cell] = 0.0; return; }
    const double *hc = h + cell - k;
    const double b = u[6];
    double zeu = hc[0] + hc[1], ztop = zeu;
    for (int i = m3d::kEuphotic; i < k; i++) ztop += hc[i];
    double zbot = ztop + hc[k];
    double rt = ztop / zeu, rb = zbot / zeu;
    double gt = -log(rt) * pow(rt, -b);
    double gb = (k == L - 1) ? 0.0 : -log(rb) * pow(rb, -b);
    mfrac_b[cell] = (gt - gb) / hc[k];
}

template <typename T>
cudaError_t upload_vec(m3d_ctx *c, const T **dst, const std::vector<T> &v)
{
    void *p = nullptr;
    cudaError_t e = m3d_alloc(c, &p, sizeof(T) * (v.empty() ? 1 : v.size()));
    if (e != cudaSuccess) return e;
    *dst = (const T *)p;
    if (v.empty()) return cudaSuccess;
    return cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
}

void free_owned(m3d_ctx *c, void *p)
{
    if (!p) return;
    for (size_t i = 0; i < c->allocs.size(); i++)
        if (c->allocs[i] == p) { c->allocs.erase(c->allocs.begin() + i); break; }
    cudaFree(p);
}

}  // namespace

m3d_status setup_adjoint(m3d_ctx *c, const AdjointSetup &in)
{
    c->adj_ok = 0;
    c->adj_stream_ok = 0;
    if (c->model != M3D_MODEL_NDOP || c->nsub != 1) return M3D_OK;
    const m3d_grid *g = in.g;
    const m3d_matrices *mt = in.mt;
    const int n = g->n;
    const int *rp = mt->exp_rowptr, *ci = mt->exp_colidx;
    // the explicit pattern must be structurally symmetric: entry (i, k) <-> (k, i)
    std::vector<int> posT(mt->nnz);
    for (int i = 0; i < n; i++)
        for (int p = rp[i]; p < rp[i + 1]; p++) {
            int k = ci[p];
            const int *b = ci + rp[k], *e = ci + rp[k + 1];
            const int *f = std::lower_bound(b, e, i);
            if (f == e || *f != i) return M3D_OK;       // not symmetric: no adjoint
            posT[p] = (int)(f - ci);
        }
    // transposed explicit values in the forward slice layout: slot (row i, entry p) holds A[k][i]
    const long long spn = c->P.sp_mstride;
    std::vector<double> a((size_t)(spn * c->nmonth), 0.0), d((size_t)(spn * c->nmonth), 0.0);
    const std::vector<int> &sp_len = *in.sp_len, &sp_off = *in.sp_off, &rows = *in.sp_rows_flat;
    for (size_t s = 0; s < sp_len.size(); s++)
        for (int l = 0; l < 32; l++) {
            int r = rows[s * 32 + l];
            if (r < 0) continue;
            int nr = rp[r + 1] - rp[r];
            for (int q = 0; q < nr; q++) {
                size_t idx = ((size_t)sp_off[s] + q) * 32 + l;
                int pt = posT[rp[r] + q];
                for (int m = 0; m < c->nmonth; m++) {
                    double a0 = mt->exp_val[(size_t)m * mt->nnz + pt];
                    double a1 = mt->exp_val[(size_t)((m + 1) % c->nmonth) * mt->nnz + pt];
                    a[(size_t)m * spn + idx] = a0;
                    d[(size_t)m * spn + idx] = a1 - a0;
                }
            }
        }
    StepParams PT = c->P;
    PT.use_tri = 0;                 // the forward Thomas factors are not the transposed operator's
    cudaError_t e = upload_vec(c, &PT.sp_a, a);
    if (e == cudaSuccess) e = upload_vec(c, &PT.sp_d, d);
    // transposed dense blocks in the forward block layout: lane (row r of column cc) holds B[k][r]
    const long long bkn = c->P.bk_mstride;
    std::vector<double> bb((size_t)(bkn * c->nmonth), 0.0), bd((size_t)(bkn * c->nmonth), 0.0);
    const std::vector<int> &bk_len = *in.bk_len, &bk_off = *in.bk_off, &brows = *in.bk_rows_flat;
    const std::vector<int> &cell_col = *in.cell_col;
    const std::vector<long long> &blk_off = *in.blk_off;
    for (size_t s = 0; s < bk_len.size() && e == cudaSuccess; s++)
        for (int l = 0; l < 32; l++) {
            int r = brows[s * 32 + l];
            if (r < 0) continue;
            int cc = cell_col[r];
            int L = g->col_start[cc + 1] - g->col_start[cc], rr = r - g->col_start[cc];
            for (int k = 0; k < L; k++) {
                size_t idx = ((size_t)bk_off[s] + k) * 32 + l;
                size_t src = (size_t)blk_off[cc] + (size_t)k * L + rr;          // B[k][rr]
                for (int m = 0; m < c->nmonth; m++) {
                    double b0 = mt->imp_blk[(size_t)m * in.s_imp + src];
                    double b1 = mt->imp_blk[(size_t)((m + 1) % c->nmonth) * in.s_imp + src];
                    bb[(size_t)m * bkn + idx] = b0;
                    bd[(size_t)m * bkn + idx] = b1 - b0;
                }
            }
        }
    if (e == cudaSuccess) e = upload_vec(c, &PT.bk_b, bb);
    if (e == cudaSuccess) e = upload_vec(c, &PT.bk_d, bd);
    m3d::ResidentParams RT = c->R;
    RT.sp_b = nullptr;              // the reverse sweep applies transposed operators
    // Thomas factors of M^T: the transposed blocks are the inverses of M^T
    if (e == cudaSuccess && c->tri_ok) {
        std::vector<double> tri((size_t)c->nmonth * 3 * n, 0.0), blk;
        bool ok = true;
        for (int m = 0; m < c->nmonth && ok; m++)
            for (int cc = 0; cc < g->ncol && ok; cc++) {
                int L = g->col_start[cc + 1] - g->col_start[cc], s0 = g->col_start[cc];
                blk.assign((size_t)L * L, 0.0);
                const double *B = mt->imp_blk + (size_t)m * in.s_imp + blk_off[cc];
                for (int r = 0; r < L; r++)
                    for (int k = 0; k < L; k++) blk[(size_t)r * L + k] = B[(size_t)k * L + r];
                double *base = tri.data() + (size_t)m * 3 * n;
                ok = tridiagonal_factors(blk.data(), L, base + s0, base + n + s0, base + 2 * (size_t)n + s0);
            }
        if (ok) {
            for (int m = 0; m < c->nmonth; m++)
                thomas_backsubstitution_form(tri.data() + (size_t)m * 3 * n, n, g->col_start, g->ncol);
            const double *tri_dev = nullptr;
            e = upload_vec(c, &tri_dev, tri);
            RT.tri = tri_dev;
            c->adj_tri_ok = ok;
        }
    }
    // per-tile column lists
    std::vector<int> col_list, col_off(c->ntiles + 1, 0);
    const std::vector<int> &bounds = *in.bounds;
    for (int t = 0; t < c->ntiles; t++) {
        int cell0 = g->col_start[bounds[t]];
        for (int cc = bounds[t]; cc < bounds[t + 1]; cc++)
            col_list.push_back((g->col_start[cc] - cell0) | ((g->col_start[cc + 1] - g->col_start[cc]) << 16));
        col_off[t + 1] = (int)col_list.size();
    }
    m3d::AdjointParams A{};
    if (e == cudaSuccess) e = upload_vec(c, &A.col_list, col_list);
    if (e == cudaSuccess) e = upload_vec(c, &A.col_off, col_off);
    void *p = nullptr;
    if (e == cudaSuccess) e = m3d_alloc(c, &p, sizeof(double) * n);
    A.mfrac_b = (const double *)p;
    c->mfrac_b = (double *)p;
    if (e == cudaSuccess) e = m3d_alloc(c, &p, sizeof(double) * 8 * c->ntiles);
    A.ubar_part = (double *)p;
    A.zc = c->zc;
    if (e != cudaSuccess) return fail(c, M3D_ERR_CUDA, "adjoint set-up: %s", cudaGetErrorString(e));
    // kernels: the same shared-memory layouts as the forward resident kernels with two tracers
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, c->device);
    const void *kd = (const void *)k_year_adjoint<false>, *kt = (const void *)k_year_adjoint<true>;
    int occ = 0;
    c->adj_smem_dense = c->resident_smem;
    c->adj_smem_tri = c->resident_tri_smem;
    c->adj_dense_ok = 0;
    if (c->adj_smem_dense <= (size_t)prop.sharedMemPerBlockOptin &&
        cudaFuncSetAttribute(kd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->adj_smem_dense) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kd, m3d::kThreads, c->adj_smem_dense) == cudaSuccess)
        c->adj_dense_ok = (long long)occ * prop.multiProcessorCount >= c->ntiles;
    if (c->adj_tri_ok) {
        occ = 0;
        if (!(c->adj_smem_tri <= (size_t)prop.sharedMemPerBlockOptin &&
              cudaFuncSetAttribute(kt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->adj_smem_tri) == cudaSuccess &&
              cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kt, m3d::kThreads, c->adj_smem_tri) == cudaSuccess &&
              (long long)occ * prop.multiProcessorCount >= c->ntiles))
            c->adj_tri_ok = 0;
    }
    // streaming sweep: operators from global memory; in shared memory the tile's cotangent
    // (2 components), the export scratch (2) and the per-column scratch (1)
    {
        const void *ks = (const void *)k_year_adjoint_stream;
        c->adj_smem_stream = sizeof(double) * 5 * (size_t)c->zmax;
        occ = 0;
        if (c->adj_smem_stream <= (size_t)prop.sharedMemPerBlockOptin &&
            cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->adj_smem_stream) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ks, m3d::kThreads, c->adj_smem_stream) == cudaSuccess)
            c->adj_stream_ok = (long long)occ * prop.multiProcessorCount >= c->ntiles;
    }
    cudaGetLastError();
    c->PT = PT;
    c->RTadj = RT;
    c->A = A;
    c->adj_ok = (c->adj_dense_ok || c->adj_tri_ok) && c->resident_ok;
    return M3D_OK;
}

namespace {

// One forward resident launch over ns steps from j0, keeping every state: traj[0] must hold
// the interleaved state of step j0; traj[s] receives the state of step j0 + s.
m3d_status forward_segment(m3d_ctx *c, bool tri, double *traj, long long len, int j0, int ns)
{
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->S.flags, 0, sizeof(int) * c->ntiles, c->stream));
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->S.status, 0, sizeof(int) * 4, c->stream));
    StepParams P = c->P;
    m3d::ResidentParams R = c->R;
    m3d::SyncParams S = c->S;
    long long stride = len;
    int period = ns + 1;
    void *args[] = {&P, &R, &S, &traj, &stride, &period, &j0, &ns};
    CUDA_OR_FAIL(c, cudaLaunchCooperativeKernel((const void *)(tri ? c->rk.year_tri : c->rk.year), dim3(c->ntiles),
                                                dim3(m3d::kThreads), args,
                                                tri ? c->resident_tri_smem : c->resident_smem, c->stream));
    return M3D_OK;
}

// The forward segment without the resident kernel: one step launch per step in the caller's
// layout, each state interleaved into the trajectory (traj[0] holds the segment's start).
m3d_status forward_segment_stream(m3d_ctx *c, double *traj, long long len, int j0, int ns)
{
    const int nb = (c->n + 255) / 256;
    double *ya = c->ybuf[0], *yb = c->ybuf[1];
    for (int s = 0; s < ns; s++) {
        c->rk.from_interleaved<<<nb, 256, 0, c->stream>>>(c->n, traj + (size_t)s * len, ya);
        CUDA_OR_FAIL(c, cudaGetLastError());
        m3d_status st = m3d_step_device(c, (j0 + s) % c->nstep, ya, yb);
        if (st != M3D_OK) return st;
        c->rk.to_interleaved<<<nb, 256, 0, c->stream>>>(c->n, yb, traj + (size_t)(s + 1) * len);
        CUDA_OR_FAIL(c, cudaGetLastError());
    }
    return M3D_OK;
}

m3d_status adjoint_segment_stream(m3d_ctx *c, const double *traj, long long len, const double *ybar_in, double *out,
                                  double *zb0, double *zb1, int j0, int ns)
{
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->S.flags, 0, sizeof(int) * c->ntiles, c->stream));
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->S.status, 0, sizeof(int) * 4, c->stream));
    StepParams PT = c->PT;
    m3d::ResidentParams RT = c->RTadj;
    m3d::SyncParams S = c->S;
    m3d::AdjointParams A = c->A;
    long long stride = len;
    void *args[] = {&PT, &RT, &S, &A, &traj, &stride, &ybar_in, &out, &zb0, &zb1, &j0, &ns};
    CUDA_OR_FAIL(c, cudaLaunchCooperativeKernel((const void *)k_year_adjoint_stream, dim3(c->ntiles),
                                                dim3(m3d::kThreads), args, c->adj_smem_stream, c->stream));
    return M3D_OK;
}

m3d_status adjoint_segment(m3d_ctx *c, bool tri, const double *traj, long long len, const double *ybar_in,
                           double *out, double *zb0, double *zb1, int j0, int ns)
{
    m3d_status st = m3d_adjoint_step_operators(c);
    if (st != M3D_OK) return st;
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->S.flags, 0, sizeof(int) * c->ntiles, c->stream));
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->S.status, 0, sizeof(int) * 4, c->stream));
    StepParams PT = c->PT;
    m3d::ResidentParams RT = c->RTadj;
    m3d::SyncParams S = c->S;
    m3d::AdjointParams A = c->A;
    long long stride = len;
    void *args[] = {&PT, &RT, &S, &A, &traj, &stride, &ybar_in, &out, &zb0, &zb1, &j0, &ns};
    CUDA_OR_FAIL(c, cudaLaunchCooperativeKernel(tri ? (const void *)k_year_adjoint<true> : (const void *)k_year_adjoint<false>,
                                                dim3(c->ntiles), dim3(m3d::kThreads), args,
                                                tri ? c->adj_smem_tri : c->adj_smem_dense, c->stream));
    return M3D_OK;
}

}  // namespace

m3d_status AdjointSweep::begin(m3d_ctx *ctx, int ckpt_every)
{
    c = ctx;
    stream = c->adj_stream_ok && (!c->adj_ok || c->adj_force_stream);
    if (!c->adj_ok && !stream)
        return fail(c, M3D_ERR_UNSUPPORTED,
                    "adjoint year map: needs the PO4-DOP model with one internal step, a structurally "
                    "symmetric explicit pattern, and a tile that fits on the GPU");
    K = ckpt_every > 0 ? std::min(ckpt_every, c->nstep) : std::min(240, c->nstep);
    nseg = (c->nstep + K - 1) / K;
    tri = !stream && c->implicit_form == M3D_IMPLICIT_TRIDIAGONAL && c->adj_tri_ok && c->tri_resident_ok;
    if (!stream && !tri && !c->adj_dense_ok)
        return fail(c, M3D_ERR_UNSUPPORTED, "adjoint year map: the dense form does not fit");
    len = (long long)c->ntr * c->n;
    const size_t vb = sizeof(double) * (size_t)len;
    const size_t sizes[4] = {vb * (size_t)(K + 1), vb * (size_t)(nseg + 1), vb * 2, vb * 2};
    double **bufs[4] = {&traj, &chk, &zb, &yb};
    for (int b = 0; b < 4; b++) {
        void *p = nullptr;
        cudaError_t e = m3d_alloc(c, &p, sizes[b]);
        if (e != cudaSuccess) {
            release();
            return fail(c, M3D_ERR_CUDA, "adjoint year map: %s (%zu bytes)", cudaGetErrorString(e), sizes[b]);
        }
        *bufs[b] = (double *)p;
    }
    held = -1;
    launches = 0;
    forward_steps = 0;
    reverse_sweeps = 0;
    return M3D_OK;
}

void AdjointSweep::release()
{
    if (!c) return;
    free_owned(c, traj);
    free_owned(c, chk);
    free_owned(c, zb);
    free_owned(c, yb);
    traj = chk = zb = yb = nullptr;
    held = -1;
}

// Recompute segment seg from its checkpoint into traj (all its states kept).
static m3d_status recompute_segment(AdjointSweep &A, int seg)
{
    m3d_ctx *c = A.c;
    const size_t vb = sizeof(double) * (size_t)A.len;
    const int j0 = seg * A.K, ns = std::min(A.K, c->nstep - j0);
    CUDA_OR_FAIL(c, cudaMemcpyAsync(A.traj, A.chk + (size_t)seg * A.len, vb, cudaMemcpyDeviceToDevice, c->stream));
    m3d_status st = A.stream ? forward_segment_stream(c, A.traj, A.len, j0, ns)
                             : forward_segment(c, A.tri, A.traj, A.len, j0, ns);
    if (st != M3D_OK) return st;
    A.launches += A.stream ? 3LL * ns : 1;
    A.forward_steps += ns;
    A.held = seg;
    return M3D_OK;
}

m3d_status AdjointSweep::forward(const double *y0, const double *u)
{
    const size_t vb = sizeof(double) * (size_t)len;
    m3d_status st = m3d_set_params(c, u, cudaMemcpyDeviceToDevice);
    if (st != M3D_OK) return st;
    st = m3d_prologue(c);
    if (st != M3D_OK) return st;
    const int nb = (c->n + 255) / 256;
    k_martin_b<<<nb, 256, 0, c->stream>>>(c->n, c->cell_kl, c->h, c->u_dev, c->mfrac_b);
    c->rk.to_interleaved<<<nb, 256, 0, c->stream>>>(c->n, y0, chk);
    CUDA_OR_FAIL(c, cudaGetLastError());
    launches += 3;
    // one checkpoint per segment; traj ends holding the last segment
    for (int seg = 0; seg < nseg; seg++) {
        st = recompute_segment(*this, seg);
        if (st != M3D_OK) return st;
        const int ns = std::min(K, c->nstep - seg * K);
        CUDA_OR_FAIL(c, cudaMemcpyAsync(chk + (size_t)(seg + 1) * len, traj + (size_t)ns * len, vb,
                                        cudaMemcpyDeviceToDevice, c->stream));
    }
    return M3D_OK;
}

m3d_status AdjointSweep::reverse(const double *ybar1, double *ybar0, double *ubar_host)
{
    const int nb = (c->n + 255) / 256;
    double *ya = yb, *ybn = yb + len;
    c->rk.to_interleaved<<<nb, 256, 0, c->stream>>>(c->n, ybar1, ya);
    CUDA_OR_FAIL(c, cudaGetLastError());
    launches += 1;
    double ub[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    std::vector<double> part((size_t)8 * c->ntiles);
    m3d_status st = M3D_OK;
    for (int seg = nseg - 1; seg >= 0; seg--) {
        const int j0 = seg * K, ns = std::min(K, c->nstep - j0);
        if (held != seg) {
            st = recompute_segment(*this, seg);
            if (st != M3D_OK) return st;
        }
        st = stream ? adjoint_segment_stream(c, traj, len, ya, ybn, zb, zb + len, j0, ns)
                    : adjoint_segment(c, tri, traj, len, ya, ybn, zb, zb + len, j0, ns);
        if (st != M3D_OK) return st;
        launches += 1;
        CUDA_OR_FAIL(c, cudaMemcpyAsync(c->status_host, c->S.status, sizeof(int) * 4, cudaMemcpyDeviceToHost, c->stream));
        CUDA_OR_FAIL(c, cudaMemcpyAsync(part.data(), c->A.ubar_part, sizeof(double) * part.size(),
                                        cudaMemcpyDeviceToHost, c->stream));
        st = metos3d_sync(c);
        if (st != M3D_OK) return st;
        for (int t = 0; t < c->ntiles; t++)
            for (int k = 0; k < 7; k++) ub[k] += part[(size_t)t * 8 + k];
        std::swap(ya, ybn);
    }
    c->rk.from_interleaved<<<nb, 256, 0, c->stream>>>(c->n, ya, ybar0);
    CUDA_OR_FAIL(c, cudaGetLastError());
    launches += 1;
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    if (ubar_host)
        for (int k = 0; k < 7; k++) ubar_host[k] = ub[k];
    reverse_sweeps++;
    return M3D_OK;
}

extern "C" m3d_status metos3d_year_adjoint(m3d_ctx *c, const double *y0, const double *u, const double *ybar1,
                                           double *ybar0, double *ubar_host, int ckpt_every)
{
    if (!c) return fail(nullptr, M3D_ERR_ARG, "metos3d_year_adjoint: null context");
    if (!y0 || !u || !ybar1 || !ybar0) return fail(c, M3D_ERR_ARG, "metos3d_year_adjoint: null pointer");
    if (c->ens) {
        // N, PO4-DOP-PHY and NPZD-DOP: the reverse sweep of the context's one-member ensemble
        m3d_status st = m3d_set_params(c, u, cudaMemcpyDeviceToDevice);
        if (st == M3D_OK) st = m3d_ens_sync_params(c);
        if (st != M3D_OK) return st;
        st = metos3d_ensemble_year_adjoint(c->ens, y0, ybar1, ybar0, ubar_host, ckpt_every);
        if (st != M3D_OK) return fail(c, st, "%s", metos3d_ensemble_last_error(c->ens));
        c->last_launches = metos3d_ensemble_last_launch_count(c->ens);
        return M3D_OK;
    }
    AdjointSweep A;
    m3d_status st = A.begin(c, ckpt_every);
    if (st == M3D_OK) st = A.forward(y0, u);
    if (st == M3D_OK) st = A.reverse(ybar1, ybar0, ubar_host);
    // prologue, Martin gradient, three layout passes; per segment a forward (one launch, or
    // three per step when streaming) and a reverse launch; the last segment is not recomputed
    if (st == M3D_OK) c->last_launches = (int)A.launches;
    A.release();
    return st;
}
