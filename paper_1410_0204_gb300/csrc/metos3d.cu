// metos3d.cu -- the C ABI of include/metos3d.h: context set-up (validation and device
// layouts), the TMM step and year map (Metos3D, arXiv:1410.0204, Sections 3 and 4),
// diagnostics and the model-interface entry of Section 5.2.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "metos3d.h"
#include "tmm_kernels.cuh"
#include "tmm_resident.cuh"
#include "context.h"
#include "adjoint.h"


// ------------------------------------------------------------------------------ kernels
namespace {

template <int NTR, int MODEL>
__global__ void __launch_bounds__(m3d::kThreads, 1) k_step(StepParams P, int j, const double *y,
                                                        double *yn)
{
    extern __shared__ double smem[];
    m3d::step_tile<NTR, MODEL, false>(P, blockIdx.x, j, y, yn, smem);
}

template <int NTR, int MODEL>
__global__ void __launch_bounds__(m3d::kThreads, 1) k_year(StepParams P, m3d::SyncParams S, double *buf0,
                                                        double *buf1, int j0, int nsteps)
{
    extern __shared__ double smem[];
    if (S.skip && *(volatile const int *)S.skip) return;
    m3d::year_persistent<NTR, MODEL>(P, S, buf0, buf1, j0, nsteps, smem);
}

template <int NTR, int MODEL, bool TRI>
__global__ void __launch_bounds__(m3d::kThreads, 1) k_year_resident(StepParams P, m3d::ResidentParams R,
                                                                 m3d::SyncParams S, double *base, long long stride,
                                                                 int period, int j0, int nsteps)
{
    if (S.skip && *(volatile const int *)S.skip) return;
    m3d::year_resident<NTR, MODEL, TRI>(P, R, S, base, stride, period, j0, nsteps);
}

// Per-step explicit operators: out[j][i] = sp_a[m0(j)][i] + w_j sp_d[m0(j)][i], as one fused
// multiply-add, the same one the year kernel otherwise evaluates for every entry and step
// (Section 4: the explicit matrix of step j interpolated linearly between the monthly means).
// Grid: blockIdx.y = step j, blocks along x stride over the slot-lanes.
__global__ void k_step_operators(long long spn, const double *__restrict__ sp_a, const double *__restrict__ sp_d,
                                 const int *__restrict__ m0tab, const double *__restrict__ wtab,
                                 double *__restrict__ out)
{
    const int j = blockIdx.y;
    const double w = wtab[j];
    const double *a = sp_a + (long long)m0tab[j] * spn, *d = sp_d + (long long)m0tab[j] * spn;
    double *o = out + (long long)j * spn;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < spn; i += (long long)gridDim.x * blockDim.x)
        o[i] = fma(w, __ldg(d + i), __ldg(a + i));
}

// Per-call tables of the PO4-DOP model that depend on the parameters u:
// atten = sigma_PAR exp(-k_w d) on euphotic cells, mfrac = Martin profile on aphotic cells.
__global__ void k_ndop_prologue(int n, const int *cell_kl, const double *h, const double *zc,
                                const double *u, double *atten, double *mfrac, double *qpar)
{
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell == 0) {
        qpar[m3d::kQAlpha] = u[1] * 360.0;       // alpha is given per day; time is in years
        qpar[m3d::kQSigma] = u[2];
        qpar[m3d::kQLambda] = u[3];
        qpar[m3d::kQKN] = u[4];
        qpar[m3d::kQKI] = u[5];
        qpar[m3d::kQOneMinusSigma] = 1.0 - u[2];
    }
    if (cell >= n) return;
    int kl = cell_kl[cell];
    int k = kl & 0xff, L = kl >> 8;
    double kw = u[0], b = u[6];
    bool euphotic = (L <= m3d::kEuphotic) || (k < m3d::kEuphotic);
    atten[cell] = euphotic ? m3d::kSigmaPar * exp(-zc[cell] * kw) : 0.0;
    mfrac[cell] = euphotic ? 0.0 : m3d::martin_fraction(h + cell - k, k, L, b);
}

// Insolation table I0[j][ulat] at the start of every step.
__global__ void k_insolation_table(int nstep, int nulat, const double *ulat, double *I0)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)nstep * nulat) return;
    int j = (int)(i / nulat), l = (int)(i % nulat);
    I0[i] = m3d::insolation(ulat[l], (double)j / nstep);
}

// Deterministic FP64 reductions: fixed grid, per-block partials, one final ordered sum.
constexpr int kRedBlocks = 512;

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double ws[m3d::kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += ws[i];
    return s;
}

// mode 0: sum vol[i mod n] a[i]; mode 1: sum (a[i] - b[i])^2; mode 2: count non-finite a[i]
__global__ void __launch_bounds__(m3d::kThreads) k_reduce(int mode, long long len, int n,
                                                          const double *a, const double *b,
                                                          const double *vol, double *part)
{
    double v = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
         i += (long long)gridDim.x * blockDim.x) {
        double x = a[i];
        if (mode == 0) v += vol[i % n] * x;
        else if (mode == 1) { double d = x - b[i]; v += d * d; }
        else v += isfinite(x) ? 0.0 : 1.0;
    }
    double s = block_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_reduce_final(int nblocks, const double *part, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nblocks; i++) s += part[i];
        out[0] = s;
    }
}

// The model interface of Section 5.2 on one column (one thread per layer).
__global__ void k_bgc_column(int model, double dt, double insol, double ice, int nlayer,
                             const double *h, const double *d, const double *y, double *ybgc,
                             const double *u, int nsub)
{
    __shared__ double ek[M3D_MAX_LAYERS];
    int k = threadIdx.x;
    if (model == m3d::kModelNone) {
        for (int i = k; i < 2 * nlayer; i += blockDim.x) ybgc[i] = 0.0;
        return;
    }
    const double kw = u[0], alpha = u[1] * 360.0, sigma = u[2], lambda = u[3], KN = u[4];
    const double KI = u[5], b = u[6];
    const double ds = dt / nsub;
    const int L = nlayer;
    const double Isurf = insol * m3d::kSigmaPar * (1.0 - ice);
    if (L <= m3d::kEuphotic) {
        if (k == 0) {
            double I[m3d::kEuphotic], dN[m3d::kEuphotic], dD[m3d::kEuphotic];
            for (int kk = 0; kk < L; kk++) I[kk] = Isurf * exp(-d[kk] * kw);
            m3d::ndop_shallow_column(L, h, y, y + L, I, alpha, sigma, lambda, KN, KI, ds, nsub, dN, dD);
            for (int kk = 0; kk < L; kk++) { ybgc[kk] = dN[kk]; ybgc[L + kk] = dD[kk]; }
        }
        return;
    }
    if (k < m3d::kEuphotic) {
        double dN, dD, fsum;
        m3d::ndop_euphotic(y[k], y[L + k], Isurf * exp(-d[k] * kw), alpha, sigma, lambda, KN, KI,
                           ds, nsub, dN, dD, fsum);
        ybgc[k] = dN;
        ybgc[L + k] = dD;
        ek[k] = (1.0 - sigma) * fsum * h[k];
    }
    __syncthreads();
    if (k >= m3d::kEuphotic && k < L) {
        double dN, dD;
        m3d::ndop_aphotic(y[L + k], ek[0] + ek[1], m3d::martin_fraction(h, k, L, b), lambda, ds,
                          nsub, dN, dD);
        ybgc[k] = dN;
        ybgc[L + k] = dD;
    }
}


year_kernel_t pick_year_kernel(int model, int ntr)
{
    if (model == m3d::kModelNdop) return ntr == 2 ? k_year<2, m3d::kModelNdop> : nullptr;
    switch (ntr) {
    case 1: return k_year<1, m3d::kModelNone>;
    case 2: return k_year<2, m3d::kModelNone>;
    case 3: return k_year<3, m3d::kModelNone>;
    case 4: return k_year<4, m3d::kModelNone>;
    case 5: return k_year<5, m3d::kModelNone>;
    case 6: return k_year<6, m3d::kModelNone>;
    case 7: return k_year<7, m3d::kModelNone>;
    case 8: return k_year<8, m3d::kModelNone>;
    default: return nullptr;
    }
}


template <int NTR, int MODEL>
ResidentKernels resident_kernels()
{
    return {k_year_resident<NTR, MODEL, false>, k_year_resident<NTR, MODEL, true>, m3d::k_interleave<NTR>,
            m3d::k_deinterleave<NTR>};
}

ResidentKernels pick_resident_kernels(int model, int ntr)
{
    if (model == m3d::kModelNdop) return ntr == 2 ? resident_kernels<2, m3d::kModelNdop>() : ResidentKernels{};
    switch (ntr) {
    case 1: return resident_kernels<1, m3d::kModelNone>();
    case 2: return resident_kernels<2, m3d::kModelNone>();
    case 3: return resident_kernels<3, m3d::kModelNone>();
    case 4: return resident_kernels<4, m3d::kModelNone>();
    case 5: return resident_kernels<5, m3d::kModelNone>();
    case 6: return resident_kernels<6, m3d::kModelNone>();
    case 7: return resident_kernels<7, m3d::kModelNone>();
    case 8: return resident_kernels<8, m3d::kModelNone>();
    default: return ResidentKernels{};
    }
}

// The model with its tangent: the state (N, DOP, dN, dDOP) as four tracers.
YearVariant tangent_kernels()
{
    YearVariant V;
    V.ntr = 4;
    V.model = m3d::kModelNdopTangent;
    V.step = k_step<4, m3d::kModelNdopTangent>;
    V.year = k_year<4, m3d::kModelNdopTangent>;
    V.rk = resident_kernels<4, m3d::kModelNdopTangent>();
    return V;
}

step_kernel_t pick_step_kernel(int model, int ntr)
{
    if (model == m3d::kModelNdop) return ntr == 2 ? k_step<2, m3d::kModelNdop> : nullptr;
    switch (ntr) {
    case 1: return k_step<1, m3d::kModelNone>;
    case 2: return k_step<2, m3d::kModelNone>;
    case 3: return k_step<3, m3d::kModelNone>;
    case 4: return k_step<4, m3d::kModelNone>;
    case 5: return k_step<5, m3d::kModelNone>;
    case 6: return k_step<6, m3d::kModelNone>;
    case 7: return k_step<7, m3d::kModelNone>;
    case 8: return k_step<8, m3d::kModelNone>;
    default: return nullptr;
    }
}

}  // namespace

thread_local std::string g_init_error;

m3d_status fail(m3d_ctx *c, m3d_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_init_error = buf;
    return s;
}

namespace {

template <typename T>
cudaError_t upload(m3d_ctx *c, T **dst, const T *src, size_t count)
{
    *dst = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)dst, sizeof(T) * count);
    if (e != cudaSuccess) return e;
    c->allocs.push_back(*dst);
    if (src) return cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice);
    return cudaSuccess;
}

template <typename T>
cudaError_t upload_vec(m3d_ctx *c, const T **dst, const std::vector<T> &v)
{
    T *p = nullptr;
    cudaError_t e = upload(c, &p, v.empty() ? nullptr : v.data(), v.size());
    *dst = p;
    return e;
}

void release(m3d_ctx *c)
{
    if (!c) return;
    if (c->year_graph) cudaGraphExecDestroy(c->year_graph);
    if (c->sp_b) cudaFree(c->sp_b);
    c->sp_b = nullptr;
    if (c->spT_b) cudaFree(c->spT_b);
    c->spT_b = nullptr;
    for (void *p : c->allocs) cudaFree(p);
    if (c->red_host) cudaFreeHost(c->red_host);
    if (c->status_host) cudaFreeHost(c->status_host);
    c->allocs.clear();
}

// Build (on) or release the per-step explicit operators the resident year kernels stream.
// Synchronous.  The array holds nstep x slot-lanes doubles (16.9 GB on the 128 x 64 x 15 grid).
m3d_status set_step_operators(m3d_ctx *c, bool on)
{
    if (!on) {
        if (c->sp_b || c->spT_b) CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
        if (c->sp_b) CUDA_OR_FAIL(c, cudaFree(c->sp_b));
        if (c->spT_b) CUDA_OR_FAIL(c, cudaFree(c->spT_b));
        c->sp_b = c->spT_b = nullptr;
        c->sp_b_bytes = c->spT_b_bytes = 0;
        c->R.sp_b = c->R_tan.sp_b = c->RTadj.sp_b = nullptr;
        return M3D_OK;
    }
    if (c->sp_b) return M3D_OK;
    const long long spn = c->P.sp_mstride;
    const size_t bytes = sizeof(double) * (size_t)spn * (size_t)c->nstep;
    double *buf = nullptr;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, M3D_ERR_CUDA, "per-step explicit operators: cannot allocate %zu bytes", bytes);
    }
    const int bx = (int)std::min<long long>((spn + 255) / 256, 64);
    k_step_operators<<<dim3(bx, c->nstep), 256, 0, c->stream>>>(spn, c->P.sp_a, c->P.sp_d, c->P.m0tab, c->P.wtab, buf);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaFree(buf);
        return fail(c, M3D_ERR_CUDA, "per-step explicit operators: %s", cudaGetErrorString(e));
    }
    c->sp_b = buf;
    c->sp_b_bytes = bytes;
    c->R.sp_b = c->R_tan.sp_b = buf;
    c->R.sp_bstride = c->R_tan.sp_bstride = spn;
    return M3D_OK;
}

}  // namespace

m3d_status m3d_adjoint_step_operators(m3d_ctx *c)
{
    if (!c->sp_b || c->spT_b || !c->adj_ok) return M3D_OK;
    const long long spn = c->P.sp_mstride;
    const size_t bytes = sizeof(double) * (size_t)spn * (size_t)c->nstep;
    size_t free_b = 0, total_b = 0;
    CUDA_OR_FAIL(c, cudaMemGetInfo(&free_b, &total_b));
    if (bytes > free_b / 4) return M3D_OK;          // keep room for the sweep's trajectory
    double *buf = nullptr;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        return M3D_OK;
    }
    const int bx = (int)std::min<long long>((spn + 255) / 256, 64);
    k_step_operators<<<dim3(bx, c->nstep), 256, 0, c->stream>>>(spn, c->PT.sp_a, c->PT.sp_d, c->P.m0tab, c->P.wtab,
                                                                buf);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaFree(buf);
        return fail(c, M3D_ERR_CUDA, "transposed per-step operators: %s", cudaGetErrorString(e));
    }
    c->spT_b = buf;
    c->spT_b_bytes = bytes;
    c->RTadj.sp_b = buf;
    c->RTadj.sp_bstride = spn;
    return M3D_OK;
}

namespace {

bool all_finite(const double *p, size_t count)
{
    for (size_t i = 0; i < count; i++)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// Contiguous partition of the water columns into tiles whose largest step time is as small as
// a contiguous partition allows.  The neighbour-synchronised year kernels run at the pace of
// their slowest tile, so the partition minimises the largest tile cost (greedy packing: each
// tile takes columns while its cost stays within W, for the smallest W that needs at most
// ntiles tiles), with no tile above max_cells cells when max_cells > 0.  A column's cost is
// ntr (0.165 nnz + 1.54 L + 13.4): per tracer, its explicit entries, its cells (Thomas solves
// and source term) and a per-column share (its chains and euphotic cells), the coefficients
// of a least-squares fit of the resident kernel's per-tile step time (nanoseconds, PO4-DOP,
// 128 x 64 x 15, GB300) to those three counts.
std::vector<int> partition_columns(const m3d_grid *g, const int *rowptr, int ntr, int ntiles, int max_cells = 0)
{
    std::vector<double> work(g->ncol);
    for (int c = 0; c < g->ncol; c++) {
        const int s = g->col_start[c], e = g->col_start[c + 1], L = e - s;
        const double nnz = rowptr[e] - rowptr[s];
        work[c] = ntr * (0.165 * nnz + 1.54 * L + 13.4);
    }
    const double total = std::accumulate(work.begin(), work.end(), 0.0);
    auto greedy = [&](double W, std::vector<int> *out) {
        int tiles = 0, cells = 0;
        double acc = 0.0;
        if (out) out->assign(1, 0);
        for (int c = 0; c < g->ncol; c++) {
            const int L = g->col_start[c + 1] - g->col_start[c];
            if (c > 0 && (acc + work[c] > W || (max_cells > 0 && cells + L > max_cells))) {
                tiles++;
                if (out) out->push_back(c);
                acc = 0.0;
                cells = 0;
            }
            acc += work[c];
            cells += L;
        }
        if (out) out->push_back(g->ncol);
        return tiles + 1;
    };
    double lo = *std::max_element(work.begin(), work.end()), hi = total;
    std::vector<int> bounds;
    if (greedy(hi, nullptr) > ntiles) {      // the cell cap alone needs more tiles
        greedy(hi, &bounds);
        return bounds;
    }
    for (int it = 0; it < 60 && hi - lo > 1e-9 * hi; it++) {
        const double mid = 0.5 * (lo + hi);
        if (greedy(mid, nullptr) <= ntiles) hi = mid;
        else lo = mid;
    }
    greedy(hi, &bounds);
    return bounds;
}

// Deal the slices [s0, s1) (cost = slot count) to the warps of one tile: longest first to
// the least loaded SM sub-partition (warp w sits on sub-partition w mod 4), round robin over
// that sub-partition's warps.  Appends to wlist and woff (nwarps + 1 offsets).
void deal_slices(int s0, int s1, const std::vector<int> &len, int nwarps, std::vector<int> &wlist,
                 std::vector<int> &woff)
{
    std::vector<int> order;
    for (int s = s0; s < s1; s++) order.push_back(s);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return len[a] > len[b]; });
    const int nsub = 4;
    std::vector<long long> load(nsub, 0);
    std::vector<int> next(nsub, 0);
    std::vector<std::vector<int>> per_warp(nwarps);
    for (int s : order) {
        int g = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[g] += len[s];
        int w = g + nsub * (next[g] % (nwarps / nsub));
        next[g]++;
        per_warp[w].push_back(s);
    }
    int base = (int)wlist.size();
    for (int w = 0; w < nwarps; w++) {
        woff.push_back(base);
        wlist.insert(wlist.end(), per_warp[w].begin(), per_warp[w].end());
        base = (int)wlist.size();
    }
    woff.push_back(base);
}

// Tracer and parameter counts of the models a single context runs through a one-member
// ensemble (0 / -1 for the others).
int ensemble_backed_ntracer(int model)
{
    return model == M3D_MODEL_N ? 1 : model == M3D_MODEL_PHY ? 3 : model == M3D_MODEL_NPZD ? 5 : 0;
}
int ensemble_backed_nparam(int model)
{
    return model == M3D_MODEL_N ? 5 : model == M3D_MODEL_PHY ? 11 : model == M3D_MODEL_NPZD ? 13 : -1;
}

// A context for N, PO4-DOP-PHY or NPZD-DOP: the steps run in a one-member ensemble; the
// context keeps what its own calls need (parameters, volumes, a staging pair of states, the
// reductions).
m3d_status init_ensemble_backed(m3d_ctx **out, const m3d_grid *g, const m3d_matrices *mt, const m3d_model *md,
                                void *stream)
{
    m3d_ctx *c = new (std::nothrow) m3d_ctx();
    if (!c) return fail(nullptr, M3D_ERR_ARG, "out of host memory");
    cudaGetLastError();
    auto bail = [&](m3d_status s) {
        g_init_error = c->err;
        if (c->ens) metos3d_ensemble_free(c->ens);
        if (c->ens_tan) metos3d_ensemble_free(c->ens_tan);
        release(c);
        delete c;
        cudaGetLastError();
        return s;
    };
    cudaGetDevice(&c->device);
    c->stream = (cudaStream_t)stream;
    c->n = g->n;
    c->ncol = g->ncol;
    c->ntr = md->ntracer;
    c->nparam = md->nparam;
    c->nsub = md->nsub;
    c->nstep = md->nstep;
    c->nmonth = mt->nmonth;
    c->model = md->model_id;
    c->plan = M3D_PLAN_GRAPH;            // one launch per step, the year one CUDA graph
    std::vector<double> u0((size_t)md->nparam, 0.0);
    m3d_member mem{md->model_id, md->nparam, u0.data()};
    m3d_status st = metos3d_ensemble_init(&c->ens, g, mt, 1, &mem, md->nsub, md->nstep, stream);
    if (st != M3D_OK) {
        c->ens = nullptr;
        fail(c, st, "%s", metos3d_ensemble_last_error(nullptr));
        return bail(st);
    }
    // its tangent (exact Jacobian-vector products, Section 6): the same member with a perturbation
    st = metos3d_ensemble_init_tangent(&c->ens_tan, g, mt, 1, &mem, md->nsub, md->nstep, stream);
    if (st != M3D_OK) {
        c->ens_tan = nullptr;
        fail(c, st, "%s", metos3d_ensemble_last_error(nullptr));
        return bail(st);
    }
    c->tan_ok = 1;
    cudaError_t e;
#define UPE(...) do { e = (__VA_ARGS__); if (e != cudaSuccess) { fail(c, M3D_ERR_CUDA, "device set-up (%s): %s", #__VA_ARGS__, cudaGetErrorString(e)); return bail(M3D_ERR_CUDA); } } while (0)
    const size_t len = (size_t)c->ntr * c->n;
    UPE(upload(c, &c->tan_buf, (const double *)nullptr, 4 * len));
    UPE(upload(c, &c->u_dev, (const double *)nullptr, (size_t)std::max(1, c->nparam)));
    UPE(upload(c, &c->vol, g->vol, (size_t)c->n));
    UPE(upload(c, &c->ybuf[0], (const double *)nullptr, 2 * len));
    c->ybuf[1] = c->ybuf[0] + len;
    c->ybuf_cap = (long long)len;
    UPE(upload(c, &c->red_part, (const double *)nullptr, (size_t)kRedBlocks));
    UPE(upload(c, &c->red_out, (const double *)nullptr, (size_t)1));
    UPE(cudaMallocHost((void **)&c->red_host, sizeof(double)));
    UPE(cudaMallocHost((void **)&c->status_host, 4 * sizeof(int)));
#undef UPE
    for (int i = 0; i < 4; i++) c->status_host[i] = 0;
    *out = c;
    return M3D_OK;
}

}  // namespace

// If the L x L row-major block B is the inverse of a tridiagonal matrix M (to 1e-11 relative),
// write the Thomas factors of M: nl[k] = -l_k, rd[k] = 1/d_k, ne[k] = -e_k / d_k, and return true.
bool tridiagonal_factors(const double *B, int L, double *nl, double *rd, double *ne)
{
    std::vector<double> a(B, B + (size_t)L * L), inv((size_t)L * L, 0.0);
    for (int i = 0; i < L; i++) inv[(size_t)i * L + i] = 1.0;
    for (int col = 0; col < L; col++) {            // Gauss-Jordan with partial pivoting
        int piv = col;
        for (int r = col + 1; r < L; r++)
            if (std::fabs(a[(size_t)r * L + col]) > std::fabs(a[(size_t)piv * L + col])) piv = r;
        if (a[(size_t)piv * L + col] == 0.0) return false;
        if (piv != col)
            for (int k = 0; k < L; k++) {
                std::swap(a[(size_t)piv * L + k], a[(size_t)col * L + k]);
                std::swap(inv[(size_t)piv * L + k], inv[(size_t)col * L + k]);
            }
        double p = a[(size_t)col * L + col];
        for (int k = 0; k < L; k++) { a[(size_t)col * L + k] /= p; inv[(size_t)col * L + k] /= p; }
        for (int r = 0; r < L; r++) {
            if (r == col) continue;
            double f = a[(size_t)r * L + col];
            if (f == 0.0) continue;
            for (int k = 0; k < L; k++) {
                a[(size_t)r * L + k] -= f * a[(size_t)col * L + k];
                inv[(size_t)r * L + k] -= f * inv[(size_t)col * L + k];
            }
        }
    }
    for (int i = 0; i < L; i++) {
        double rowmax = 0.0;
        for (int k = 0; k < L; k++) rowmax = std::max(rowmax, std::fabs(inv[(size_t)i * L + k]));
        for (int k = 0; k < L; k++)
            if (std::abs(i - k) > 1 && std::fabs(inv[(size_t)i * L + k]) > 1e-11 * rowmax) return false;
    }
    double dprev = 0.0;
    for (int k = 0; k < L; k++) {
        double l = k > 0 ? inv[(size_t)k * L + k - 1] / dprev : 0.0;
        double d = inv[(size_t)k * L + k] - (k > 0 ? l * inv[(size_t)(k - 1) * L + k] : 0.0);
        if (!(d > 0.0) || !std::isfinite(d)) return false;
        nl[k] = -l;
        rd[k] = 1.0 / d;
        ne[k] = k + 1 < L ? -inv[(size_t)k * L + k + 1] * rd[k] : 0.0;
        dprev = d;
    }
    return true;
}

// Checks of a grid and its matrices shared by metos3d_init and metos3d_ensemble_init.
m3d_status m3d_validate_inputs(const m3d_grid *g, const m3d_matrices *mt, std::string &why)
{
    char buf[256];
    auto bad = [&](const char *fmt, auto... args) {
        snprintf(buf, sizeof buf, fmt, args...);
        why = buf;
        return M3D_ERR_ARG;
    };
    if (!g || !mt) return bad("%s", "null grid or matrices");
    if (g->n <= 0 || g->ncol <= 0 || !g->col_start || !g->h || !g->zc || !g->vol || !g->lat)
        return bad("%s", "grid: bad sizes or null arrays");
    if (g->col_start[0] != 0 || g->col_start[g->ncol] != g->n)
        return bad("%s", "grid: col_start must run from 0 to n");
    long long s_imp = 0;
    for (int c = 0; c < g->ncol; c++) {
        int L = g->col_start[c + 1] - g->col_start[c];
        if (L < 1 || L > M3D_MAX_LAYERS) return bad("grid: column %d has %d layers (1..%d allowed)", c, L, M3D_MAX_LAYERS);
        if (!(g->lat[c] >= -90.0 && g->lat[c] <= 90.0)) return bad("grid: latitude of column %d out of range", c);
        s_imp += (long long)L * L;
    }
    for (int i = 0; i < g->n; i++)
        if (!(g->h[i] > 0.0) || !std::isfinite(g->h[i]) || !std::isfinite(g->zc[i]) || !std::isfinite(g->vol[i]))
            return bad("grid: bad h, zc or vol at cell %d", i);
    if (mt->nmonth < 1 || mt->nnz < g->n || !mt->exp_rowptr || !mt->exp_colidx || !mt->exp_val || !mt->imp_blk)
        return bad("%s", "matrices: bad sizes or null arrays");
    if (mt->s_imp != s_imp) return bad("matrices: s_imp is %lld, the columns need %lld", mt->s_imp, s_imp);
    const int *rp = mt->exp_rowptr, *ci = mt->exp_colidx;
    if (rp[0] != 0 || rp[g->n] != mt->nnz) return bad("%s", "matrices: rowptr must run from 0 to nnz");
    for (int i = 0; i < g->n; i++) {
        if (rp[i + 1] < rp[i]) return bad("matrices: rowptr decreases at row %d", i);
        // checked before the row's indices are read: an entry beyond nnz would read past them
        if (rp[i + 1] > mt->nnz) return bad("matrices: rowptr exceeds nnz at row %d", i);
        for (int p = rp[i]; p < rp[i + 1]; p++) {
            if (ci[p] < 0 || ci[p] >= g->n) return bad("matrices: column index out of range in row %d", i);
            if (p > rp[i] && ci[p] <= ci[p - 1]) return bad("matrices: row %d is not sorted or has duplicates", i);
        }
    }
    if (!all_finite(mt->exp_val, (size_t)mt->nmonth * mt->nnz) || !all_finite(mt->imp_blk, (size_t)mt->nmonth * s_imp))
        return bad("%s", "matrices: non-finite values");
    return M3D_OK;
}

// Rewrite the third Thomas factor of every column from -e_k/d_k to -e_k/d_{k+1} (0 at the
// bottom): the resident kernels back-substitute u_k = d_k y_k, u_k = g_k - (e_k/d_{k+1}) u_{k+1},
// one multiply-add per layer, and scale by 1/d_k when they blend the months.
void thomas_backsubstitution_form(double *tri_month, int n, const int *col_start, int ncol)
{
    const double *rd = tri_month + n;
    double *ne = tri_month + 2 * (size_t)n;
    for (int c = 0; c < ncol; c++)
        for (int i = col_start[c]; i + 1 < col_start[c + 1]; i++) ne[i] = ne[i] * rd[i + 1] / rd[i];
}

// ------------------------------------------------------------------------------ C ABI
extern "C" {

const char *metos3d_last_error(const m3d_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

m3d_status metos3d_info(const m3d_ctx *ctx, int *n, int *ncol, int *ntracer, int *nstep)
{
    if (!ctx) return fail(nullptr, M3D_ERR_ARG, "metos3d_info: null context");
    if (n) *n = ctx->n;
    if (ncol) *ncol = ctx->ncol;
    if (ntracer) *ntracer = ctx->ntr;
    if (nstep) *nstep = ctx->nstep;
    return M3D_OK;
}

long long metos3d_last_launch_count(const m3d_ctx *ctx) { return ctx ? ctx->last_launches : -1; }

void metos3d_free(m3d_ctx *ctx)
{
    if (!ctx) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    release(ctx);
    for (cudaEvent_t e : ctx->kev)
        if (e) cudaEventDestroy(e);
    if (ctx->ens) metos3d_ensemble_free(ctx->ens);
    if (ctx->ens_tan) metos3d_ensemble_free(ctx->ens_tan);
    cudaSetDevice(prev);
    delete ctx;
}

m3d_status metos3d_set_stream(m3d_ctx *ctx, void *stream)
{
    if (!ctx) return fail(nullptr, M3D_ERR_ARG, "metos3d_set_stream: null context");
    ctx->stream = (cudaStream_t)stream;
    if (ctx->ens) metos3d_ensemble_set_stream(ctx->ens, stream);
    if (ctx->ens_tan) metos3d_ensemble_set_stream(ctx->ens_tan, stream);
    return M3D_OK;
}

m3d_status metos3d_init(m3d_ctx **out, const m3d_grid *g, const m3d_matrices *mt,
                        const m3d_model *md, void *stream)
{
    if (!out) return fail(nullptr, M3D_ERR_ARG, "metos3d_init: out is null");
    *out = nullptr;
    if (!g || !mt || !md) return fail(nullptr, M3D_ERR_ARG, "metos3d_init: null grid, matrices or model");
    // ---- validation
    std::string why;
    if (m3d_validate_inputs(g, mt, why) != M3D_OK) return fail(nullptr, M3D_ERR_ARG, "%s", why.c_str());
    long long s_imp = mt->s_imp;
    const int *rp = mt->exp_rowptr, *ci = mt->exp_colidx;
    if (md->nstep <= 0 || md->nsub < 1)
        return fail(nullptr, M3D_ERR_ARG, "model: nstep and nsub must be positive");
    if (md->model_id == M3D_MODEL_NDOP) {
        if (md->ntracer != 2 || md->nparam != 7)
            return fail(nullptr, M3D_ERR_ARG, "model: PO4-DOP needs 2 tracers and 7 parameters");
    } else if (md->model_id == M3D_MODEL_NONE) {
        if (md->ntracer < 1 || md->ntracer > M3D_MAX_TRACERS || md->nparam < 0)
            return fail(nullptr, M3D_ERR_ARG, "model: 1..%d tracers for the transport-only model", M3D_MAX_TRACERS);
    } else if (ensemble_backed_ntracer(md->model_id) > 0) {
        if (md->ntracer != ensemble_backed_ntracer(md->model_id) || md->nparam != ensemble_backed_nparam(md->model_id))
            return fail(nullptr, M3D_ERR_ARG, "model: model %d needs %d tracers and %d parameters", md->model_id,
                        ensemble_backed_ntracer(md->model_id), ensemble_backed_nparam(md->model_id));
        return init_ensemble_backed(out, g, mt, md, stream);
    } else {
        return fail(nullptr, M3D_ERR_UNSUPPORTED, "model: unknown model_id %d", md->model_id);
    }

    m3d_ctx *c = new (std::nothrow) m3d_ctx();
    if (!c) return fail(nullptr, M3D_ERR_ARG, "out of host memory");
    cudaGetLastError();                 // an earlier failed call must not be reported here
    auto bail = [&](m3d_status s) {
        g_init_error = c->err;
        release(c);
        delete c;
        cudaGetLastError();             // nor this one's by a later call
        return s;
    };
    cudaGetDevice(&c->device);
    c->stream = (cudaStream_t)stream;
    c->n = g->n;
    c->ncol = g->ncol;
    c->ntr = md->ntracer;
    c->nparam = md->nparam;
    c->nsub = md->nsub;
    c->nstep = md->nstep;
    c->nmonth = mt->nmonth;
    c->model = md->model_id;
    c->step_kernel = pick_step_kernel(c->model, c->ntr);
    c->year_kernel = pick_year_kernel(c->model, c->ntr);
    c->rk = pick_resident_kernels(c->model, c->ntr);
    if (!c->step_kernel || !c->year_kernel) {
        fail(c, M3D_ERR_UNSUPPORTED, "no step kernel for model %d with %d tracers", c->model, c->ntr);
        return bail(M3D_ERR_UNSUPPORTED);
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) {
        fail(c, M3D_ERR_CUDA, "cudaGetDeviceProperties failed");
        return bail(M3D_ERR_CUDA);
    }

    // ---- tiles of whole columns
    // one tile (CTA of 16 warps) per SM by default; METOS3D_TILES_PER_SM overrides it for tuning
    int tiles_per_sm = 1;
    if (const char *env = getenv("METOS3D_TILES_PER_SM")) tiles_per_sm = std::max(1, std::min(8, atoi(env)));
    int ntarget = std::min(g->ncol, tiles_per_sm * prop.multiProcessorCount);
    {
        // a tile's state must fit in shared memory: more (smaller) tiles on very large grids
        const double per_cell = sizeof(double) * (double)(c->ntr + 2);
        const long long need = (long long)(1.25 * g->n * per_cell / (double)prop.sharedMemPerBlockOptin) + 1;
        ntarget = (int)std::min<long long>(g->ncol, std::max<long long>(ntarget, need));
    }
    // PO4-DOP contexts also run the tangent, whose tile holds four components: cap the tile so
    // that they fit in shared memory (binding only on very large grids)
    int max_cells = 0;
    if (md->model_id == M3D_MODEL_NDOP)
        max_cells = (int)(((long long)prop.sharedMemPerBlockOptin - 2048) / (sizeof(double) * (2 * c->ntr + 2)));
    std::vector<int> bounds = partition_columns(g, rp, c->ntr, ntarget, max_cells);
    int ntiles = (int)bounds.size() - 1;
    c->ntiles = ntiles;

    std::vector<Tile> tiles(ntiles);
    std::vector<int> sp_len, sp_off, sp_row, sp_col;
    std::vector<int> bk_len, bk_off, bk_row, bk_cb, bk_L;
    std::vector<int> eu_list, ap_list, sh_list;
    int sp_slots = 0, bk_slots = 0, zmax = 0;
    // first pass: the slice structure; values are filled per month afterwards
    struct SliceRef { int tile_cell0; std::vector<int> rows; };
    std::vector<int> sp_rows_flat, bk_rows_flat;   // global row per (slice, lane), -1 if empty
    for (int t = 0; t < ntiles; t++) {
        int c0 = bounds[t], c1 = bounds[t + 1];
        int cell0 = g->col_start[c0], cell1 = g->col_start[c1];
        int nc = cell1 - cell0;
        zmax = std::max(zmax, nc);
        Tile &T = tiles[t];
        T.cell0 = cell0;
        T.ncell = nc;
        // explicit slices: rows by decreasing nonzero count
        std::vector<int> rows(nc);
        std::iota(rows.begin(), rows.end(), cell0);
        std::stable_sort(rows.begin(), rows.end(), [&](int a, int b) {
            return (rp[a + 1] - rp[a]) > (rp[b + 1] - rp[b]);
        });
        T.sp0 = (int)sp_len.size();
        for (int s0 = 0; s0 < nc; s0 += 32) {
            int len = 0;
            for (int l = 0; l < 32; l++) {
                int r = s0 + l < nc ? rows[s0 + l] : -1;
                sp_rows_flat.push_back(r);
                sp_row.push_back(r >= 0 ? r - cell0 : -1);
                if (r >= 0) len = std::max(len, rp[r + 1] - rp[r]);
            }
            sp_len.push_back(len);
            sp_off.push_back(sp_slots);
            sp_slots += len;
        }
        T.sp1 = (int)sp_len.size();
        // implicit slices: rows by decreasing column depth
        std::vector<int> colL(nc), colB(nc);
        for (int cc = c0; cc < c1; cc++)
            for (int i = g->col_start[cc]; i < g->col_start[cc + 1]; i++) {
                colL[i - cell0] = g->col_start[cc + 1] - g->col_start[cc];
                colB[i - cell0] = g->col_start[cc] - cell0;
            }
        std::vector<int> brow(nc);
        std::iota(brow.begin(), brow.end(), 0);
        std::stable_sort(brow.begin(), brow.end(), [&](int a, int b) { return colL[a] > colL[b]; });
        T.bk0 = (int)bk_len.size();
        for (int s0 = 0; s0 < nc; s0 += 32) {
            int len = 0;
            for (int l = 0; l < 32; l++) {
                int r = s0 + l < nc ? brow[s0 + l] : -1;
                bk_rows_flat.push_back(r >= 0 ? r + cell0 : -1);
                bk_row.push_back(r);
                bk_cb.push_back(r >= 0 ? colB[r] : 0);
                bk_L.push_back(r >= 0 ? colL[r] : 0);
                if (r >= 0) len = std::max(len, colL[r]);
            }
            bk_len.push_back(len);
            bk_off.push_back(bk_slots);
            bk_slots += len;
        }
        T.bk1 = (int)bk_len.size();
        // source-term work lists: euphotic cells of deep columns and the first cell of each
        // shallow column (which then runs whole on one thread); aphotic cells
        T.eu0 = (int)eu_list.size();
        T.ap0 = (int)ap_list.size();
        T.sh0 = (int)sh_list.size();
        for (int cc = c0; cc < c1; cc++) {
            int L = g->col_start[cc + 1] - g->col_start[cc];
            int base = g->col_start[cc] - cell0;
            if (L <= m3d::kEuphotic && md->nsub > 1) {
                eu_list.push_back(base);                 // the whole column on one thread
            } else {
                for (int k = 0; k < std::min(L, m3d::kEuphotic); k++) eu_list.push_back(base + k);
                if (L <= m3d::kEuphotic) sh_list.push_back(base + L - 1);
            }
        }
        for (int cc = c0; cc < c1; cc++) {
            int L = g->col_start[cc + 1] - g->col_start[cc];
            int base = g->col_start[cc] - cell0;
            for (int k = m3d::kEuphotic; k < L; k++) ap_list.push_back(base + k);
        }
        T.eu1 = (int)eu_list.size();
        T.ap1 = (int)ap_list.size();
        T.sh1 = (int)sh_list.size();
    }
    c->zmax = zmax;

    // neighbour tiles: those this tile reads from and those that read from it
    std::vector<int> cell_tile(g->n);
    for (int t = 0; t < ntiles; t++)
        for (int i = tiles[t].cell0; i < tiles[t].cell0 + tiles[t].ncell; i++) cell_tile[i] = t;
    std::vector<std::vector<int>> nbr(ntiles);
    for (int t = 0; t < ntiles; t++)
        for (int r = tiles[t].cell0; r < tiles[t].cell0 + tiles[t].ncell; r++)
            for (int p = rp[r]; p < rp[r + 1]; p++) {
                int o = cell_tile[ci[p]];
                if (o != t) { nbr[t].push_back(o); nbr[o].push_back(t); }
            }
    std::vector<int> dep_off(ntiles + 1, 0), dep_idx;
    for (int t = 0; t < ntiles; t++) {
        std::sort(nbr[t].begin(), nbr[t].end());
        nbr[t].erase(std::unique(nbr[t].begin(), nbr[t].end()), nbr[t].end());
        dep_idx.insert(dep_idx.end(), nbr[t].begin(), nbr[t].end());
        dep_off[t + 1] = (int)dep_idx.size();
    }

    // month and weight of every step (the weight needs a division: do it once here)
    std::vector<int> m0tab(c->nstep);
    std::vector<double> wtab(c->nstep);
    for (int j = 0; j < c->nstep; j++) m3d::month_weights(j, c->nstep, c->nmonth, m0tab[j], wtab[j]);

    // column block offsets and per-cell tables
    std::vector<long long> blk_off(g->ncol + 1, 0);
    for (int cc = 0; cc < g->ncol; cc++) {
        long long L = g->col_start[cc + 1] - g->col_start[cc];
        blk_off[cc + 1] = blk_off[cc] + L * L;
    }
    std::vector<int> cell_col(g->n), cell_kl(g->n), cell_ulat(g->n);
    std::vector<double> ulat(g->lat, g->lat + g->ncol);
    std::sort(ulat.begin(), ulat.end());
    ulat.erase(std::unique(ulat.begin(), ulat.end()), ulat.end());
    c->nulat = (int)ulat.size();
    for (int cc = 0; cc < g->ncol; cc++) {
        int L = g->col_start[cc + 1] - g->col_start[cc];
        int li = (int)(std::lower_bound(ulat.begin(), ulat.end(), g->lat[cc]) - ulat.begin());
        for (int k = 0; k < L; k++) {
            int i = g->col_start[cc] + k;
            cell_col[i] = cc;
            cell_kl[i] = k | (L << 8);
            cell_ulat[i] = li;
        }
    }

    // values in slice layout, month by month: A_m and A_{m+1} - A_m
    const long long spn = (long long)sp_slots * 32, bkn = (long long)bk_slots * 32;
    std::vector<double> sp_a((size_t)(spn * c->nmonth), 0.0), sp_d((size_t)(spn * c->nmonth), 0.0);
    sp_col.assign((size_t)spn, 0);
    for (size_t s = 0; s < sp_len.size(); s++)
        for (int l = 0; l < 32; l++) {
            int r = sp_rows_flat[s * 32 + l];
            for (int q = 0; q < sp_len[s]; q++) {
                size_t idx = ((size_t)sp_off[s] + q) * 32 + l;
                if (r < 0) { sp_col[idx] = 0; continue; }
                int nr = rp[r + 1] - rp[r];
                int p = rp[r] + std::min(q, nr - 1);
                sp_col[idx] = ci[p];
                for (int m = 0; m < c->nmonth; m++) {
                    double a0 = q < nr ? mt->exp_val[(size_t)m * mt->nnz + p] : 0.0;
                    double a1 = q < nr ? mt->exp_val[(size_t)((m + 1) % c->nmonth) * mt->nnz + p] : 0.0;
                    sp_a[(size_t)m * spn + idx] = a0;
                    sp_d[(size_t)m * spn + idx] = a1 - a0;
                }
            }
        }
    std::vector<double> bk_b((size_t)(bkn * c->nmonth), 0.0), bk_d((size_t)(bkn * c->nmonth), 0.0);
    for (size_t s = 0; s < bk_len.size(); s++)
        for (int l = 0; l < 32; l++) {
            int r = bk_rows_flat[s * 32 + l];
            if (r < 0) continue;
            int cc = cell_col[r];
            int L = g->col_start[cc + 1] - g->col_start[cc];
            int rr = r - g->col_start[cc];
            for (int k = 0; k < L; k++) {
                size_t idx = ((size_t)bk_off[s] + k) * 32 + l;
                size_t src = (size_t)blk_off[cc] + (size_t)rr * L + k;
                for (int m = 0; m < c->nmonth; m++) {
                    double b0 = mt->imp_blk[(size_t)m * s_imp + src];
                    double b1 = mt->imp_blk[(size_t)((m + 1) % c->nmonth) * s_imp + src];
                    bk_b[(size_t)m * bkn + idx] = b0;
                    bk_d[(size_t)m * bkn + idx] = b1 - b0;
                }
            }
        }

    // ---- upload
    StepParams &P = c->P;
    P.n = c->n;
    P.nstep = c->nstep;
    P.nmonth = c->nmonth;
    P.nsub = c->nsub;
    P.nulat = c->nulat;
    P.zmax = c->zmax;
    P.sp_mstride = spn;
    P.bk_mstride = bkn;
    P.ds = (1.0 / c->nstep) / c->nsub;
    cudaError_t e = cudaSuccess;
#define UP(...) do { e = (__VA_ARGS__); if (e != cudaSuccess) { fail(c, M3D_ERR_CUDA, "device set-up (%s): %s", #__VA_ARGS__, cudaGetErrorString(e)); return bail(M3D_ERR_CUDA); } } while (0)
    UP(upload_vec(c, &P.tiles, tiles));
    UP(upload_vec(c, &P.sp_len, sp_len));
    UP(upload_vec(c, &P.sp_off, sp_off));
    UP(upload_vec(c, &P.sp_row, sp_row));
    UP(upload_vec(c, &P.sp_col, sp_col));
    UP(upload_vec(c, &P.sp_a, sp_a));
    UP(upload_vec(c, &P.sp_d, sp_d));
    UP(upload_vec(c, &P.bk_len, bk_len));
    UP(upload_vec(c, &P.bk_off, bk_off));
    UP(upload_vec(c, &P.bk_row, bk_row));
    UP(upload_vec(c, &P.bk_cb, bk_cb));
    UP(upload_vec(c, &P.bk_L, bk_L));
    {
        std::vector<int> spw, spwo, bkw, bkwo, spwg, spwog;
        const int nwarps = m3d::kThreads / 32;
        for (int t = 0; t < ntiles; t++) {
            deal_slices(tiles[t].sp0, tiles[t].sp1, sp_len, nwarps, spw, spwo);
            deal_slices(tiles[t].bk0, tiles[t].bk1, bk_len, nwarps, bkw, bkwo);
            // the resident kernel's explicit group (its other warps evaluate the source term)
            deal_slices(tiles[t].sp0, tiles[t].sp1, sp_len, m3d::kSpThreads / 32, spwg, spwog);
        }
        UP(upload_vec(c, &P.sp_wlist, spw));
        UP(upload_vec(c, &P.sp_woff, spwo));
        UP(upload_vec(c, &P.sp_wlist_g, spwg));
        UP(upload_vec(c, &P.sp_woff_g, spwog));
        UP(upload_vec(c, &P.bk_wlist, bkw));
        UP(upload_vec(c, &P.bk_woff, bkwo));
    }
    UP(upload_vec(c, &P.bk_b, bk_b));
    UP(upload_vec(c, &P.bk_d, bk_d));
    UP(upload_vec(c, &P.m0tab, m0tab));
    UP(upload_vec(c, &P.wtab, wtab));
    UP(upload_vec(c, &P.eu_list, eu_list));
    P.n_eu = (int)eu_list.size();
    UP(upload_vec(c, &P.ap_list, ap_list));
    UP(upload_vec(c, &P.sh_list, sh_list));
    {
        const int *p_off = nullptr, *p_idx = nullptr;
        UP(upload_vec(c, &p_off, dep_off));
        UP(upload_vec(c, &p_idx, dep_idx));
        c->S.dep_off = p_off;
        c->S.dep_idx = p_idx;
        UP(upload(c, &c->S.flags, (const int *)nullptr, (size_t)ntiles));
        UP(upload(c, &c->S.status, (const int *)nullptr, (size_t)4));
        UP(cudaMemset(c->S.status, 0, 4 * sizeof(int)));
        UP(cudaMallocHost((void **)&c->status_host, 4 * sizeof(int)));
        memset(c->status_host, 0, 4 * sizeof(int));
        c->S.timeout_ns = 2000000000ULL;      // 2 s; one step takes microseconds
        c->S.withhold_tile = -1;
    }
    UP(upload(c, &c->qpar, (const double *)nullptr, (size_t)m3d::kQCount));
    UP(cudaMemset(c->qpar, 0, sizeof(double) * m3d::kQCount));
    P.qpar = c->qpar;
    UP(upload_vec(c, &P.cell_kl, cell_kl));
    UP(upload_vec(c, &P.cell_ulat, cell_ulat));
    c->cell_kl = const_cast<int *>(P.cell_kl);
    UP(upload(c, &c->h, g->h, (size_t)c->n));
    UP(upload(c, &c->zc, g->zc, (size_t)c->n));
    UP(upload(c, &c->vol, g->vol, (size_t)c->n));
    P.h = c->h;
    UP(upload(c, &c->atten, (const double *)nullptr, (size_t)c->n));
    UP(upload(c, &c->mfrac, (const double *)nullptr, (size_t)c->n));
    P.atten = c->atten;
    P.mfrac = c->mfrac;
    UP(upload(c, &c->u_dev, (const double *)nullptr, (size_t)std::max(1, c->nparam)));
    const size_t ybuf_len = (size_t)(c->model == M3D_MODEL_NDOP ? 2 * c->ntr : c->ntr) * c->n;
    UP(upload(c, &c->ybuf[0], (const double *)nullptr, 2 * ybuf_len));   // one allocation: the
    c->ybuf[1] = c->ybuf[0] + ybuf_len;                                   // resident kernel strides
    c->ybuf_cap = (long long)ybuf_len;
    UP(upload(c, &c->red_part, (const double *)nullptr, (size_t)kRedBlocks));
    UP(upload(c, &c->red_out, (const double *)nullptr, (size_t)1));
    UP(cudaMallocHost((void **)&c->red_host, sizeof(double)));
    UP(cudaMemset(c->atten, 0, sizeof(double) * c->n));
    UP(cudaMemset(c->mfrac, 0, sizeof(double) * c->n));
    UP(cudaMemset(c->u_dev, 0, sizeof(double) * std::max(1, c->nparam)));
    // insolation table at the start of every step
    double *ulat_dev = nullptr, *I0 = nullptr;
    UP(upload(c, &ulat_dev, ulat.data(), ulat.size()));
    UP(upload(c, &I0, (const double *)nullptr, (size_t)c->nstep * c->nulat));
    {
        long long tot = (long long)c->nstep * c->nulat;
        k_insolation_table<<<(unsigned)((tot + 255) / 256), 256>>>(c->nstep, c->nulat, ulat_dev, I0);
        UP(cudaGetLastError());
        UP(cudaDeviceSynchronize());
    }
    P.I0tab = I0;
    c->smem_bytes = sizeof(double) * (size_t)(c->ntr + 2) * c->zmax;
    if (c->smem_bytes > (size_t)prop.sharedMemPerBlockOptin) {
        fail(c, M3D_ERR_UNSUPPORTED, "a tile of %d cells does not fit in shared memory", c->zmax);
        return bail(M3D_ERR_UNSUPPORTED);
    }
    if (c->smem_bytes > 48 * 1024) {
        UP(cudaFuncSetAttribute((const void *)c->step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)c->smem_bytes));
        UP(cudaFuncSetAttribute((const void *)c->year_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)c->smem_bytes));
    }
    {
        // the persistent year kernels need every tile resident at once
        int per_sm = 0, coop = 0;
        UP(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)c->year_kernel, m3d::kThreads,
                                                         c->smem_bytes));
        UP(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device));
        c->persistent_ok = coop && (long long)per_sm * prop.multiProcessorCount >= ntiles;
        // resident plan: the tile's month of matrices in shared memory
        std::vector<m3d::ResidentTile> rt(ntiles);
        int sp_max = 0, bk_max = 0;
        for (int t = 0; t < ntiles; t++) {
            const Tile &T = tiles[t];
            int sp_first = T.sp0 < T.sp1 ? sp_off[T.sp0] : 0, sp_slots = 0;
            for (int q = T.sp0; q < T.sp1; q++) sp_slots += sp_len[q];
            int bk_first = T.bk0 < T.bk1 ? bk_off[T.bk0] : 0, bk_slots_t = 0;
            for (int q = T.bk0; q < T.bk1; q++) bk_slots_t += bk_len[q];
            rt[t].sp_base = (long long)sp_first * 32;
            rt[t].sp_n = sp_slots * 32;
            rt[t].bk_base = (long long)bk_first * 32;
            rt[t].bk_n = bk_slots_t * 32;
            rt[t].pad0 = rt[t].pad1 = 0;
            sp_max = std::max(sp_max, rt[t].sp_n);
            bk_max = std::max(bk_max, rt[t].bk_n);
        }
        m3d::ResidentLayout Ly = m3d::resident_layout(c->ntr, sp_max, bk_max, c->zmax, false);
        m3d::ResidentLayout Lt = m3d::resident_layout(c->ntr, sp_max, bk_max, c->zmax, true);
        c->resident_smem = (size_t)Ly.total;
        c->resident_tri_smem = (size_t)Lt.total;
        const m3d::ResidentTile *rt_dev = nullptr;
        UP(upload_vec(c, &rt_dev, rt));
        c->R.rt = rt_dev;
        c->R.sp_max = sp_max;
        c->R.bk_max = bk_max;
        c->R_tan.rt = rt_dev;
        c->R_tan.sp_max = sp_max;
        c->R_tan.bk_max = bk_max;
        // tridiagonal form of the implicit blocks, when every one of them has it
        {
            std::vector<double> tri((size_t)c->nmonth * 3 * c->n, 0.0);
            bool ok = true;
            for (int m = 0; m < c->nmonth && ok; m++)
                for (int cc = 0; cc < g->ncol && ok; cc++) {
                    int L = g->col_start[cc + 1] - g->col_start[cc], s0 = g->col_start[cc];
                    double *base = tri.data() + (size_t)m * 3 * c->n;
                    ok = tridiagonal_factors(mt->imp_blk + (size_t)m * s_imp + blk_off[cc], L, base + s0,
                                             base + c->n + s0, base + 2 * (size_t)c->n + s0);
                }
            c->tri_ok = ok;
            if (ok) {
                for (int m = 0; m < c->nmonth; m++)
                    thomas_backsubstitution_form(tri.data() + (size_t)m * 3 * c->n, c->n, g->col_start, g->ncol);
                const double *tri_dev = nullptr;
                UP(upload_vec(c, &tri_dev, tri));
                c->R.tri = tri_dev;
                c->R.tri_mstride = 3LL * c->n;
                c->R_tan.tri = tri_dev;
                c->R_tan.tri_mstride = 3LL * c->n;
                // (column, tracer) chains of the streaming kernels' Thomas part, deepest first
                if (c->ntr <= 2) {
                    std::vector<int> tch, tch_off(ntiles + 1, 0);
                    for (int t = 0; t < ntiles; t++) {
                        int c0 = bounds[t], c1 = bounds[t + 1], cell0 = g->col_start[c0];
                        std::vector<int> cols;
                        for (int cc = c0; cc < c1; cc++) cols.push_back(cc);
                        std::stable_sort(cols.begin(), cols.end(), [&](int a, int b) {
                            return (g->col_start[a + 1] - g->col_start[a]) > (g->col_start[b + 1] - g->col_start[b]);
                        });
                        for (int cc : cols)
                            for (int tr = 0; tr < c->ntr; tr++)
                                tch.push_back(m3d::pack_chain(g->col_start[cc] - cell0,
                                                              g->col_start[cc + 1] - g->col_start[cc], tr, 0));
                        tch_off[t + 1] = (int)tch.size();
                    }
                    UP(upload_vec(c, &P.tchains, tch));
                    UP(upload_vec(c, &P.tchain_off, tch_off));
                    P.tri = tri_dev;
                    P.tri_mstride = 3LL * c->n;
                    c->tri_stream_ok = 1;
                }
                // Thomas chains (column, component, month) per tile, deepest columns first; the
                // model with its tangent has twice the components
                for (int variant = 0; variant < 2; variant++) {
                    const int ncomp = variant == 0 ? c->ntr : 2 * c->ntr;
                    if (variant == 1 && c->model != M3D_MODEL_NDOP) break;
                    std::vector<int> chains, chain_off(ntiles + 1, 0);
                    for (int t = 0; t < ntiles; t++) {
                        int c0 = bounds[t], c1 = bounds[t + 1], cell0 = g->col_start[c0];
                        std::vector<int> cols;
                        for (int cc = c0; cc < c1; cc++) cols.push_back(cc);
                        std::stable_sort(cols.begin(), cols.end(), [&](int a, int b) {
                            return (g->col_start[a + 1] - g->col_start[a]) > (g->col_start[b + 1] - g->col_start[b]);
                        });
                        for (int cc : cols)
                            for (int h = 0; h < 2; h++)
                                for (int tr = 0; tr < ncomp; tr++)
                                    chains.push_back(m3d::pack_chain(g->col_start[cc] - cell0,
                                                                     g->col_start[cc + 1] - g->col_start[cc], tr, h));
                        chain_off[t + 1] = (int)chains.size();
                    }
                    const int *ch_dev = nullptr, *choff_dev = nullptr;
                    UP(upload_vec(c, &ch_dev, chains));
                    UP(upload_vec(c, &choff_dev, chain_off));
                    m3d::ResidentParams &RR = variant == 0 ? c->R : c->R_tan;
                    RR.chains = ch_dev;
                    RR.chain_off = choff_dev;
                }
            }
        }
        if (coop && c->rk.year && c->resident_smem <= (size_t)prop.sharedMemPerBlockOptin) {
            UP(cudaFuncSetAttribute((const void *)c->rk.year, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)c->resident_smem));
            int rps = 0;
            UP(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rps, (const void *)c->rk.year, m3d::kThreads,
                                                             c->resident_smem));
            c->resident_ok = (long long)rps * prop.multiProcessorCount >= ntiles;
        }
        if (coop && c->tri_ok && c->rk.year_tri && c->resident_tri_smem <= (size_t)prop.sharedMemPerBlockOptin) {
            UP(cudaFuncSetAttribute((const void *)c->rk.year_tri, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)c->resident_tri_smem));
            int rps = 0;
            UP(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rps, (const void *)c->rk.year_tri, m3d::kThreads,
                                                             c->resident_tri_smem));
            c->tri_resident_ok = (long long)rps * prop.multiProcessorCount >= ntiles;
        }
        if (c->tri_resident_ok && !c->resident_ok) c->resident_ok = 1;
        if (c->model == M3D_MODEL_NDOP && c->nsub == 1 && coop) {
            // the linearised year kernels: the forward model's tiles, layouts and shared memory
            c->rk_lin = resident_kernels<2, m3d::kModelNdopLinear>();
            int rps = 0;
            if (c->resident_smem <= (size_t)prop.sharedMemPerBlockOptin) {
                UP(cudaFuncSetAttribute((const void *)c->rk_lin.year, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)c->resident_smem));
                UP(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rps, (const void *)c->rk_lin.year, m3d::kThreads,
                                                                 c->resident_smem));
                c->lin_ok = (long long)rps * prop.multiProcessorCount >= ntiles;
            }
            if (c->tri_ok && c->resident_tri_smem <= (size_t)prop.sharedMemPerBlockOptin) {
                UP(cudaFuncSetAttribute((const void *)c->rk_lin.year_tri, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)c->resident_tri_smem));
                UP(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rps, (const void *)c->rk_lin.year_tri, m3d::kThreads,
                                                                 c->resident_tri_smem));
                c->lin_tri_ok = (long long)rps * prop.multiProcessorCount >= ntiles;
            }
        }
        c->plan = c->resident_ok ? M3D_PLAN_RESIDENT : (c->persistent_ok ? M3D_PLAN_PERSISTENT : M3D_PLAN_GRAPH);
        // the Thomas form wherever the plan in use can apply it
        const bool tri_here = c->plan == M3D_PLAN_RESIDENT ? c->tri_resident_ok : c->tri_stream_ok;
        c->implicit_form = tri_here ? M3D_IMPLICIT_TRIDIAGONAL : M3D_IMPLICIT_DENSE;
        P.use_tri = c->implicit_form == M3D_IMPLICIT_TRIDIAGONAL && c->tri_stream_ok;
        if (c->model == M3D_MODEL_NDOP) {
            // the model with its tangent: same tiles, four state components
            YearVariant &V = c->tan;
            V = tangent_kernels();
            V.smem = sizeof(double) * (size_t)(V.ntr + 2) * c->zmax;
            V.resident_smem = (size_t)m3d::resident_layout(V.ntr, sp_max, bk_max, c->zmax, false).total;
            V.resident_tri_smem = (size_t)m3d::resident_layout(V.ntr, sp_max, bk_max, c->zmax, true).total;
            int occ = 0;
            // a tile's four components must fit in shared memory (on very large grids they do
            // not, and the tangent is then unavailable for this context)
            if (V.smem <= (size_t)prop.sharedMemPerBlockOptin) {
                if (V.smem > 48 * 1024)
                    UP(cudaFuncSetAttribute((const void *)V.year, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)V.smem));
                UP(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)V.year, m3d::kThreads, V.smem));
            }
            V.persistent_ok = coop && (long long)occ * prop.multiProcessorCount >= ntiles;
            if (coop && V.resident_smem <= (size_t)prop.sharedMemPerBlockOptin) {
                UP(cudaFuncSetAttribute((const void *)V.rk.year, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)V.resident_smem));
                UP(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)V.rk.year, m3d::kThreads,
                                                                 V.resident_smem));
                V.resident_ok = (long long)occ * prop.multiProcessorCount >= ntiles;
            }
            if (coop && c->tri_ok && V.resident_tri_smem <= (size_t)prop.sharedMemPerBlockOptin) {
                UP(cudaFuncSetAttribute((const void *)V.rk.year_tri, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)V.resident_tri_smem));
                UP(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)V.rk.year_tri, m3d::kThreads,
                                                                 V.resident_tri_smem));
                V.tri_resident_ok = (long long)occ * prop.multiProcessorCount >= ntiles;
            }
            c->tan_ok = V.persistent_ok || V.resident_ok || V.tri_resident_ok;
        }
    }
    {
        AdjointSetup as{g, mt, s_imp, &sp_rows_flat, &sp_len, &sp_off, &bk_rows_flat, &bk_len, &bk_off, &bounds,
                        &cell_col, &blk_off};
        m3d_status ast = setup_adjoint(c, as);
        if (ast != M3D_OK) return bail(ast);
    }
    if (c->resident_ok) {
        // per-step explicit operators by default when they take at most an eighth of the free
        // device memory (HBM is plentiful on this GPU, FP64 issue is not)
        size_t free_b = 0, total_b = 0;
        UP(cudaMemGetInfo(&free_b, &total_b));
        const size_t need = sizeof(double) * (size_t)c->P.sp_mstride * (size_t)c->nstep;
        if (need <= free_b / 8) {
            m3d_status sst = set_step_operators(c, true);
            if (sst != M3D_OK) return bail(sst);
        }
    }
#undef UP
    *out = c;
    return M3D_OK;
}

}  // extern "C"

namespace {

// An ensemble-backed context: give its member the parameters now in c->u_dev (synchronous;
// re-tabulated only when they changed).
m3d_status ens_sync_params(m3d_ctx *c)
{
    std::vector<double> u((size_t)c->nparam);
    CUDA_OR_FAIL(c, cudaMemcpyAsync(u.data(), c->u_dev, sizeof(double) * u.size(), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    if (c->ens_u_valid && u == c->ens_u) return M3D_OK;
    m3d_status st = metos3d_ensemble_set_params(c->ens, 0, u.data());
    if (st != M3D_OK) return fail(c, st, "%s", metos3d_ensemble_last_error(c->ens));
    c->ens_u = u;
    c->ens_u_valid = 1;
    return M3D_OK;
}

// The same for the tangent ensemble of an ensemble-backed context.
m3d_status ens_tan_sync_params(m3d_ctx *c)
{
    std::vector<double> u((size_t)c->nparam);
    CUDA_OR_FAIL(c, cudaMemcpyAsync(u.data(), c->u_dev, sizeof(double) * u.size(), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    if (c->ens_tan_u_valid && u == c->ens_tan_u) return M3D_OK;
    m3d_status st = metos3d_ensemble_set_params(c->ens_tan, 0, u.data());
    if (st != M3D_OK) return fail(c, st, "%s", metos3d_ensemble_last_error(c->ens_tan));
    c->ens_tan_u = u;
    c->ens_tan_u_valid = 1;
    return M3D_OK;
}

// phi(y0) and phi'(y0) v of an ensemble-backed context by its tangent ensemble.
m3d_status ens_tangent_run(m3d_ctx *c, const double *y0, const double *v, double *phi, double *jv)
{
    m3d_status st = ens_tan_sync_params(c);
    if (st != M3D_OK) return st;
    const size_t len = (size_t)c->ntr * c->n;
    double *in = c->tan_buf, *out = c->tan_buf + 2 * len;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(in, y0, sizeof(double) * len, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(in + len, v, sizeof(double) * len, cudaMemcpyDeviceToDevice, c->stream));
    st = metos3d_ensemble_set_stream(c->ens_tan, c->stream);
    if (st == M3D_OK) st = metos3d_ensemble_year_map(c->ens_tan, in, out);
    if (st != M3D_OK) return fail(c, st, "%s", metos3d_ensemble_last_error(c->ens_tan));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(phi, out, sizeof(double) * len, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(jv, out + len, sizeof(double) * len, cudaMemcpyDeviceToDevice, c->stream));
    c->last_launches = metos3d_ensemble_last_launch_count(c->ens_tan);
    return M3D_OK;
}

// The year (or nsteps steps from j0) of an ensemble-backed context, device arrays.
m3d_status ens_run(m3d_ctx *c, int j0, int nsteps, const double *y0, double *y1)
{
    m3d_status st = ens_sync_params(c);
    if (st != M3D_OK) return st;
    st = nsteps < 0 ? metos3d_ensemble_year_map(c->ens, y0, y1) : metos3d_ensemble_steps(c->ens, j0, nsteps, y0, y1);
    if (st != M3D_OK) return fail(c, st, "%s", metos3d_ensemble_last_error(c->ens));
    c->last_launches = metos3d_ensemble_last_launch_count(c->ens);
    return M3D_OK;
}

m3d_status launch_prologue(m3d_ctx *c, const double *u)
{
    if (c->model != M3D_MODEL_NDOP) return M3D_OK;
    k_ndop_prologue<<<(c->n + 255) / 256, 256, 0, c->stream>>>(c->n, c->cell_kl, c->h, c->zc, u,
                                                               c->atten, c->mfrac, c->qpar);
    CUDA_OR_FAIL(c, cudaGetLastError());
    return M3D_OK;
}

m3d_status launch_step(m3d_ctx *c, int j, const double *y, double *yn)
{
    c->step_kernel<<<c->ntiles, m3d::kThreads, c->smem_bytes, c->stream>>>(c->P, j, y, yn);
    CUDA_OR_FAIL(c, cudaGetLastError());
    return M3D_OK;
}

// One cooperative launch of a streaming persistent year kernel for nsteps steps from j0:
// y in buf[0], result in buf[nsteps & 1].
m3d_status launch_year_persistent(m3d_ctx *c, year_kernel_t kernel, size_t smem, int j0, int nsteps)
{
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->S.flags, 0, sizeof(int) * c->ntiles, c->stream));
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->S.status, 0, sizeof(int) * 4, c->stream));
    StepParams P = c->P;
    m3d::SyncParams S = c->S;
    double *b0 = c->ybuf[0], *b1 = c->ybuf[1];
    void *args[] = {&P, &S, &b0, &b1, &j0, &nsteps};
    if (c->time_kernel) CUDA_OR_FAIL(c, cudaEventRecord(c->kev[0], c->stream));
    CUDA_OR_FAIL(c, cudaLaunchCooperativeKernel((const void *)kernel, dim3(c->ntiles), dim3(m3d::kThreads), args, smem,
                                                c->stream));
    if (c->time_kernel) {
        CUDA_OR_FAIL(c, cudaEventRecord(c->kev[1], c->stream));
        c->kev_recorded = 1;
    }
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->status_host, c->S.status, sizeof(int) * 4, cudaMemcpyDeviceToHost, c->stream));
    return M3D_OK;
}

m3d_status build_year_graph(m3d_ctx *c)
{
    cudaStream_t s = c->stream;
    bool own = false;
    if (!s) {
        // capture needs a non-legacy stream
        CUDA_OR_FAIL(c, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        own = true;
    }
    cudaStream_t saved = c->stream;
    c->stream = s;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    m3d_status st = M3D_OK;
    if (e == cudaSuccess) {
        st = launch_prologue(c, c->u_dev);
        for (int j = 0; j < c->nstep && st == M3D_OK; j++)
            st = launch_step(c, j, c->ybuf[j & 1], c->ybuf[(j + 1) & 1]);
        e = cudaStreamEndCapture(s, &graph);
    }
    c->stream = saved;
    if (own) cudaStreamDestroy(s);
    if (st != M3D_OK) { if (graph) cudaGraphDestroy(graph); return st; }
    if (e != cudaSuccess) return fail(c, M3D_ERR_CUDA, "year graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->year_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(c, M3D_ERR_CUDA, "year graph instantiate: %s", cudaGetErrorString(e));
    c->year_result_buf = c->nstep & 1;
    return M3D_OK;
}

// Run the year from ybuf[0] (u already in u_dev) and copy the result to `out`.
m3d_status run_year_from_ybuf(m3d_ctx *c, double *out, cudaMemcpyKind kind)
{
    size_t len = sizeof(double) * (size_t)c->ntr * c->n;
    if (c->plan == M3D_PLAN_RESIDENT) {
        m3d_status st = launch_prologue(c, c->u_dev);
        if (st != M3D_OK) return st;
        const int nb = (c->n + 255) / 256;
        // the year runs on the interleaved state: start in ybuf[1]
        c->rk.to_interleaved<<<nb, 256, 0, c->stream>>>(c->n, c->ybuf[0], c->ybuf[1]);
        CUDA_OR_FAIL(c, cudaGetLastError());
        CUDA_OR_FAIL(c, cudaMemsetAsync(c->S.flags, 0, sizeof(int) * c->ntiles, c->stream));
        CUDA_OR_FAIL(c, cudaMemsetAsync(c->S.status, 0, sizeof(int) * 4, c->stream));
        StepParams P = c->P;
        m3d::ResidentParams R = c->R;
        m3d::SyncParams S = c->S;
        double *b0 = c->ybuf[1], *b1 = c->ybuf[0];
        long long stride = -c->ybuf_cap;                    // y_s = ybuf[1] - (s mod 2) cap
        int period = 2, j0 = 0, nsteps = c->nstep;
        void *args[] = {&P, &R, &S, &b0, &stride, &period, &j0, &nsteps};
        const bool tri = c->implicit_form == M3D_IMPLICIT_TRIDIAGONAL && c->tri_resident_ok;
        if (c->time_kernel) CUDA_OR_FAIL(c, cudaEventRecord(c->kev[0], c->stream));
        CUDA_OR_FAIL(c, cudaLaunchCooperativeKernel((const void *)(tri ? c->rk.year_tri : c->rk.year), dim3(c->ntiles),
                                                    dim3(m3d::kThreads), args,
                                                    tri ? c->resident_tri_smem : c->resident_smem, c->stream));
        if (c->time_kernel) {
            CUDA_OR_FAIL(c, cudaEventRecord(c->kev[1], c->stream));
            c->kev_recorded = 1;
        }
        CUDA_OR_FAIL(c, cudaMemcpyAsync(c->status_host, c->S.status, sizeof(int) * 4, cudaMemcpyDeviceToHost,
                                        c->stream));
        double *res = (nsteps & 1) ? b1 : b0;
        double *other = (nsteps & 1) ? b0 : b1;
        if (kind == cudaMemcpyDeviceToDevice) {
            c->rk.from_interleaved<<<nb, 256, 0, c->stream>>>(c->n, res, out);
            CUDA_OR_FAIL(c, cudaGetLastError());
        } else {
            c->rk.from_interleaved<<<nb, 256, 0, c->stream>>>(c->n, res, other);
            CUDA_OR_FAIL(c, cudaGetLastError());
            CUDA_OR_FAIL(c, cudaMemcpyAsync(out, other, len, kind, c->stream));
        }
        c->last_launches = (c->model == M3D_MODEL_NDOP ? 1 : 0) + 3;
        return M3D_OK;
    }
    if (c->plan == M3D_PLAN_PERSISTENT) {
        m3d_status st = launch_prologue(c, c->u_dev);
        if (st != M3D_OK) return st;
        st = launch_year_persistent(c, c->year_kernel, c->smem_bytes, 0, c->nstep);
        if (st != M3D_OK) return st;
        CUDA_OR_FAIL(c, cudaMemcpyAsync(out, c->ybuf[c->nstep & 1], len, kind, c->stream));
        c->last_launches = (c->model == M3D_MODEL_NDOP ? 1 : 0) + 1;
    } else {
        CUDA_OR_FAIL(c, cudaGraphLaunch(c->year_graph, c->stream));
        CUDA_OR_FAIL(c, cudaMemcpyAsync(out, c->ybuf[c->year_result_buf], len, kind, c->stream));
        c->last_launches = (c->model == M3D_MODEL_NDOP ? 1 : 0) + c->nstep;
    }
    return M3D_OK;
}

// The year of the model with its tangent from ybuf[0] = [y; v] ([4][n]); result [phi; phi' v]
// into out_y and out_v (device).  Uses the resident plan where it fits, else the streaming
// persistent kernel.
m3d_status run_year_tangent(m3d_ctx *c, double *out_y, double *out_v)
{
    const YearVariant &V = c->tan;
    const size_t half = sizeof(double) * (size_t)c->ntr * c->n;
    m3d_status st = launch_prologue(c, c->u_dev);
    if (st != M3D_OK) return st;
    const bool tri = c->implicit_form == M3D_IMPLICIT_TRIDIAGONAL && V.tri_resident_ok;
    const bool resident = c->plan == M3D_PLAN_RESIDENT && (tri || V.resident_ok);
    if (resident) {
        const int nb = (c->n + 255) / 256;
        V.rk.to_interleaved<<<nb, 256, 0, c->stream>>>(c->n, c->ybuf[0], c->ybuf[1]);
        CUDA_OR_FAIL(c, cudaGetLastError());
        CUDA_OR_FAIL(c, cudaMemsetAsync(c->S.flags, 0, sizeof(int) * c->ntiles, c->stream));
        CUDA_OR_FAIL(c, cudaMemsetAsync(c->S.status, 0, sizeof(int) * 4, c->stream));
        StepParams P = c->P;
        m3d::ResidentParams R = c->R_tan;
        m3d::SyncParams S = c->S;
        double *b0 = c->ybuf[1], *b1 = c->ybuf[0];
        long long stride = -c->ybuf_cap;
        int period = 2, j0 = 0, nsteps = c->nstep;
        void *args[] = {&P, &R, &S, &b0, &stride, &period, &j0, &nsteps};
        CUDA_OR_FAIL(c, cudaLaunchCooperativeKernel((const void *)(tri ? V.rk.year_tri : V.rk.year), dim3(c->ntiles),
                                                    dim3(m3d::kThreads), args,
                                                    tri ? V.resident_tri_smem : V.resident_smem, c->stream));
        CUDA_OR_FAIL(c, cudaMemcpyAsync(c->status_host, c->S.status, sizeof(int) * 4, cudaMemcpyDeviceToHost,
                                        c->stream));
        double *res = (nsteps & 1) ? b1 : b0, *other = (nsteps & 1) ? b0 : b1;
        V.rk.from_interleaved<<<nb, 256, 0, c->stream>>>(c->n, res, other);
        CUDA_OR_FAIL(c, cudaGetLastError());
        CUDA_OR_FAIL(c, cudaMemcpyAsync(out_y, other, half, cudaMemcpyDeviceToDevice, c->stream));
        CUDA_OR_FAIL(c, cudaMemcpyAsync(out_v, (char *)other + half, half, cudaMemcpyDeviceToDevice, c->stream));
        c->last_launches = 4;
        return M3D_OK;
    }
    if (!V.persistent_ok) return fail(c, M3D_ERR_UNSUPPORTED, "the tangent year kernel does not fit on this GPU");
    st = launch_year_persistent(c, V.year, V.smem, 0, c->nstep);
    if (st != M3D_OK) return st;
    double *res = c->ybuf[c->nstep & 1];
    CUDA_OR_FAIL(c, cudaMemcpyAsync(out_y, res, half, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(out_v, (char *)res + half, half, cudaMemcpyDeviceToDevice, c->stream));
    c->last_launches = 2;
    return M3D_OK;
}

// The linearised year from ybuf[0] = v ([2][n]) about the trajectory recorded in fn; result
// phi'(y) v into out (device).  Resident plan, the forward model's tiles and layouts.
m3d_status run_year_linear(m3d_ctx *c, const double *fn, double *out)
{
    const bool tri = c->implicit_form == M3D_IMPLICIT_TRIDIAGONAL && c->lin_tri_ok && c->tri_resident_ok;
    if (!(tri || (c->lin_ok && c->implicit_form == M3D_IMPLICIT_DENSE)))
        return fail(c, M3D_ERR_UNSUPPORTED, "the linearised year kernel does not serve this context's plan");
    m3d_status st = launch_prologue(c, c->u_dev);
    if (st != M3D_OK) return st;
    const int nb = (c->n + 255) / 256;
    c->rk.to_interleaved<<<nb, 256, 0, c->stream>>>(c->n, c->ybuf[0], c->ybuf[1]);
    CUDA_OR_FAIL(c, cudaGetLastError());
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->S.flags, 0, sizeof(int) * c->ntiles, c->stream));
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->S.status, 0, sizeof(int) * 4, c->stream));
    StepParams P = c->P;
    P.fn_in = fn;
    P.fn_out = nullptr;
    m3d::ResidentParams R = c->R;
    m3d::SyncParams S = c->S;
    double *b0 = c->ybuf[1], *b1 = c->ybuf[0];
    long long stride = -c->ybuf_cap;
    int period = 2, j0 = 0, nsteps = c->nstep;
    void *args[] = {&P, &R, &S, &b0, &stride, &period, &j0, &nsteps};
    if (c->time_kernel) CUDA_OR_FAIL(c, cudaEventRecord(c->kev[0], c->stream));
    CUDA_OR_FAIL(c, cudaLaunchCooperativeKernel((const void *)(tri ? c->rk_lin.year_tri : c->rk_lin.year),
                                                dim3(c->ntiles), dim3(m3d::kThreads), args,
                                                tri ? c->resident_tri_smem : c->resident_smem, c->stream));
    if (c->time_kernel) {
        CUDA_OR_FAIL(c, cudaEventRecord(c->kev[1], c->stream));
        c->kev_recorded = 1;
    }
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->status_host, c->S.status, sizeof(int) * 4, cudaMemcpyDeviceToHost, c->stream));
    double *res = (nsteps & 1) ? b1 : b0;
    c->rk.from_interleaved<<<nb, 256, 0, c->stream>>>(c->n, res, out);
    CUDA_OR_FAIL(c, cudaGetLastError());
    c->last_launches = 4;
    return M3D_OK;
}

m3d_status reduce(m3d_ctx *c, int mode, const double *a, const double *b, double *out)
{
    long long len = (long long)c->ntr * c->n;
    k_reduce<<<kRedBlocks, m3d::kThreads, 0, c->stream>>>(mode, len, c->n, a, b, c->vol, c->red_part);
    CUDA_OR_FAIL(c, cudaGetLastError());
    k_reduce_final<<<1, 32, 0, c->stream>>>(kRedBlocks, c->red_part, c->red_out);
    CUDA_OR_FAIL(c, cudaGetLastError());
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->red_host, c->red_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    *out = *c->red_host;
    return M3D_OK;
}

}  // namespace

extern "C" {

m3d_status metos3d_step(m3d_ctx *c, int j, const double *y_in, double *y_out, const double *u)
{
    if (!c) return fail(nullptr, M3D_ERR_ARG, "metos3d_step: null context");
    if (j < 0 || j >= c->nstep) return fail(c, M3D_ERR_ARG, "metos3d_step: j = %d outside [0, %d)", j, c->nstep);
    if (!y_in || !y_out || (c->nparam > 0 && !u)) return fail(c, M3D_ERR_ARG, "metos3d_step: null pointer");
    size_t len = sizeof(double) * (size_t)c->ntr * c->n;
    const char *a = (const char *)y_in, *b = (const char *)y_out;
    if (a < b + len && b < a + len) return fail(c, M3D_ERR_ARG, "metos3d_step: y_in and y_out overlap");
    if (c->nparam > 0)
        CUDA_OR_FAIL(c, cudaMemcpyAsync(c->u_dev, u, sizeof(double) * c->nparam, cudaMemcpyDeviceToDevice, c->stream));
    if (c->ens) return ens_run(c, j, 1, y_in, y_out);
    m3d_status st = launch_prologue(c, c->u_dev);
    if (st != M3D_OK) return st;
    return launch_step(c, j, y_in, y_out);
}

m3d_status metos3d_year_map(m3d_ctx *c, const double *y0, double *y1, const double *u)
{
    if (!c) return fail(nullptr, M3D_ERR_ARG, "metos3d_year_map: null context");
    if (!y0 || !y1 || (c->nparam > 0 && !u)) return fail(c, M3D_ERR_ARG, "metos3d_year_map: null pointer");
    size_t len = sizeof(double) * (size_t)c->ntr * c->n;
    if (c->ens) {
        if (c->nparam > 0)
            CUDA_OR_FAIL(c, cudaMemcpyAsync(c->u_dev, u, sizeof(double) * c->nparam, cudaMemcpyDeviceToDevice, c->stream));
        return ens_run(c, 0, -1, y0, y1);
    }
    if (c->plan == 1 && !c->year_graph) {
        m3d_status st = build_year_graph(c);
        if (st != M3D_OK) return st;
    }
    if (c->nparam > 0)
        CUDA_OR_FAIL(c, cudaMemcpyAsync(c->u_dev, u, sizeof(double) * c->nparam, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->ybuf[0], y0, len, cudaMemcpyDeviceToDevice, c->stream));
    return run_year_from_ybuf(c, y1, cudaMemcpyDeviceToDevice);
}

m3d_status metos3d_year_map_host(m3d_ctx *c, const double *y0_host, double *y1_host, const double *u_host)
{
    if (!c) return fail(nullptr, M3D_ERR_ARG, "metos3d_year_map_host: null context");
    if (!y0_host || !y1_host || (c->nparam > 0 && !u_host))
        return fail(c, M3D_ERR_ARG, "metos3d_year_map_host: null pointer");
    size_t len = sizeof(double) * (size_t)c->ntr * c->n;
    if (c->ens) {
        if (c->nparam > 0)
            CUDA_OR_FAIL(c, cudaMemcpyAsync(c->u_dev, u_host, sizeof(double) * c->nparam, cudaMemcpyHostToDevice, c->stream));
        CUDA_OR_FAIL(c, cudaMemcpyAsync(c->ybuf[0], y0_host, len, cudaMemcpyHostToDevice, c->stream));
        m3d_status st = ens_run(c, 0, -1, c->ybuf[0], c->ybuf[1]);
        if (st != M3D_OK) return st;
        CUDA_OR_FAIL(c, cudaMemcpyAsync(y1_host, c->ybuf[1], len, cudaMemcpyDeviceToHost, c->stream));
        CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
        return M3D_OK;
    }
    if (c->plan == 1 && !c->year_graph) {
        m3d_status st = build_year_graph(c);
        if (st != M3D_OK) return st;
    }
    if (c->nparam > 0)
        CUDA_OR_FAIL(c, cudaMemcpyAsync(c->u_dev, u_host, sizeof(double) * c->nparam, cudaMemcpyHostToDevice, c->stream));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->ybuf[0], y0_host, len, cudaMemcpyHostToDevice, c->stream));
    m3d_status st = run_year_from_ybuf(c, y1_host, cudaMemcpyDeviceToHost);
    if (st != M3D_OK) return st;
    return metos3d_sync(c);
}

m3d_status metos3d_sync(m3d_ctx *c)
{
    if (!c) return fail(nullptr, M3D_ERR_ARG, "metos3d_sync: null context");
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    if (c->status_host[0] != 0) {
        int tile = c->status_host[1], step = c->status_host[2], copy = c->status_host[3];
        c->status_host[0] = 0;
        c->status_host[3] = 0;
        return fail(c, M3D_ERR_TIMEOUT, "year map: tile %d gave up waiting for its neighbours at step %d%s", tile, step,
                    copy ? " (and its own operator copy did not land within the bound)" : "");
    }
    return M3D_OK;
}

m3d_status metos3d_set_option(m3d_ctx *c, int option, long long value)
{
    if (!c) return fail(nullptr, M3D_ERR_ARG, "metos3d_set_option: null context");
    if (c->ens && option != M3D_OPT_WAIT_TIMEOUT_NS)
        return fail(c, M3D_ERR_UNSUPPORTED, "option %d: this model runs in a one-member ensemble (one launch per step)",
                    option);
    switch (option) {
    case M3D_OPT_YEAR_PLAN:
        if (value == M3D_PLAN_PERSISTENT && !c->persistent_ok)
            return fail(c, M3D_ERR_UNSUPPORTED, "the persistent year kernel does not fit on this GPU");
        if (value == M3D_PLAN_RESIDENT && !c->resident_ok)
            return fail(c, M3D_ERR_UNSUPPORTED, "the tiles' matrices do not fit in shared memory");
        if (value != M3D_PLAN_PERSISTENT && value != M3D_PLAN_GRAPH && value != M3D_PLAN_RESIDENT)
            return fail(c, M3D_ERR_ARG, "bad plan");
        c->plan = (int)value;
        return M3D_OK;
    case M3D_OPT_WAIT_TIMEOUT_NS:
        if (value <= 0) return fail(c, M3D_ERR_ARG, "timeout must be positive");
        c->S.timeout_ns = (unsigned long long)value;
        return M3D_OK;
    case M3D_OPT_IMPLICIT_FORM:
        if (value == M3D_IMPLICIT_TRIDIAGONAL && !c->tri_resident_ok && !c->tri_stream_ok)
            return fail(c, M3D_ERR_UNSUPPORTED, "the implicit blocks have no usable tridiagonal form");
        if (value == M3D_IMPLICIT_DENSE && c->plan == M3D_PLAN_RESIDENT &&
            !(c->resident_smem <= c->resident_tri_smem || c->resident_ok))
            return fail(c, M3D_ERR_UNSUPPORTED, "the dense resident kernel does not fit");
        if (value != M3D_IMPLICIT_DENSE && value != M3D_IMPLICIT_TRIDIAGONAL) return fail(c, M3D_ERR_ARG, "bad form");
        c->implicit_form = (int)value;
        c->P.use_tri = c->implicit_form == M3D_IMPLICIT_TRIDIAGONAL && c->tri_stream_ok;
        if (c->year_graph) {                 // its launches captured the previous form
            cudaGraphExecDestroy(c->year_graph);
            c->year_graph = nullptr;
        }
        return M3D_OK;
    case M3D_OPT_TEST_WITHHOLD_TILE:
        if (value < -1 || value >= c->ntiles) return fail(c, M3D_ERR_ARG, "tile out of range");
        c->S.withhold_tile = (int)value;
        return M3D_OK;
    case M3D_OPT_STEP_OPERATORS:
        if (value != 0 && value != 1) return fail(c, M3D_ERR_ARG, "step operators: 0 or 1");
        if (value == 1 && !c->resident_ok)
            return fail(c, M3D_ERR_UNSUPPORTED, "per-step operators serve the resident year kernel only");
        return set_step_operators(c, value == 1);
    case M3D_OPT_TANGENT_FORM:
        if (value != M3D_TANGENT_DUAL && value != M3D_TANGENT_LINEARISED)
            return fail(c, M3D_ERR_ARG, "tangent form: M3D_TANGENT_DUAL or M3D_TANGENT_LINEARISED");
        if (value == M3D_TANGENT_LINEARISED && (c->plan != M3D_PLAN_RESIDENT || !(c->lin_ok || c->lin_tri_ok)))
            return fail(c, M3D_ERR_UNSUPPORTED, "the linearised tangent needs PO4-DOP, one internal step and the "
                                                "resident plan");
        c->tangent_form = (int)value;
        return M3D_OK;
    case M3D_OPT_KERNEL_TIMING:
        if (value != 0 && value != 1) return fail(c, M3D_ERR_ARG, "kernel timing: 0 or 1");
        for (int i = 0; i < 2 && value == 1; i++)
            if (!c->kev[i]) CUDA_OR_FAIL(c, cudaEventCreate(&c->kev[i]));
        c->time_kernel = (int)value;
        return M3D_OK;
    case M3D_OPT_ADJOINT_PLAN:
        if (value == M3D_PLAN_PERSISTENT && !c->adj_stream_ok)
            return fail(c, M3D_ERR_UNSUPPORTED, "the streaming adjoint sweep does not fit on this GPU");
        if (value == M3D_PLAN_RESIDENT && !c->adj_ok)
            return fail(c, M3D_ERR_UNSUPPORTED, "the resident adjoint sweep does not fit on this GPU");
        if (value != M3D_PLAN_PERSISTENT && value != M3D_PLAN_RESIDENT) return fail(c, M3D_ERR_ARG, "bad adjoint plan");
        c->adj_force_stream = value == M3D_PLAN_PERSISTENT;
        return M3D_OK;
    default:
        return fail(c, M3D_ERR_ARG, "unknown option %d", option);
    }
}

long long metos3d_get_option(const m3d_ctx *c, int option)
{
    if (!c) return -1;
    switch (option) {
    case M3D_OPT_YEAR_PLAN: return c->plan;
    case M3D_OPT_WAIT_TIMEOUT_NS: return (long long)c->S.timeout_ns;
    case M3D_OPT_TEST_WITHHOLD_TILE: return c->S.withhold_tile;
    case M3D_OPT_NTILES: return c->ntiles;
    case M3D_OPT_IMPLICIT_FORM: return c->implicit_form;
    case M3D_OPT_STEP_OPERATORS: return c->sp_b != nullptr ? 1 : 0;
    case M3D_OPT_STEP_OPERATOR_BYTES: return (long long)c->sp_b_bytes;
    case M3D_OPT_KERNEL_TIMING: return c->time_kernel;
    case M3D_OPT_TANGENT_FORM: return c->tangent_form;
    case M3D_OPT_LAST_KERNEL_NS: {
        float ms = 0.0f;
        if (!c->kev_recorded || cudaEventElapsedTime(&ms, c->kev[0], c->kev[1]) != cudaSuccess) return -1;
        return (long long)((double)ms * 1e6);
    }
    case M3D_OPT_ADJOINT_PLAN:
        if (c->adj_stream_ok && (!c->adj_ok || c->adj_force_stream)) return M3D_PLAN_PERSISTENT;
        return c->adj_ok ? M3D_PLAN_RESIDENT : -1;
    default: return -1;
    }
}

m3d_status metos3d_mass(m3d_ctx *c, const double *y, double *mass)
{
    if (!c || !y || !mass) return fail(c, M3D_ERR_ARG, "metos3d_mass: null argument");
    return reduce(c, 0, y, nullptr, mass);
}

m3d_status metos3d_residual(m3d_ctx *c, const double *a, const double *b, double *norm)
{
    if (!c || !a || !b || !norm) return fail(c, M3D_ERR_ARG, "metos3d_residual: null argument");
    double s = 0.0;
    m3d_status st = reduce(c, 1, a, b, &s);
    if (st == M3D_OK) *norm = std::sqrt(s);
    return st;
}

m3d_status metos3d_check_finite(m3d_ctx *c, const double *y)
{
    if (!c || !y) return fail(c, M3D_ERR_ARG, "metos3d_check_finite: null argument");
    double bad = 0.0;
    m3d_status st = reduce(c, 2, y, nullptr, &bad);
    if (st != M3D_OK) return st;
    if (bad != 0.0) return fail(c, M3D_ERR_NONFINITE, "state holds %.0f non-finite values", bad);
    return M3D_OK;
}

m3d_status metos3d_bgc(int model_id, double t, double dt, double lat, double insol, double dayfrac,
                       double ice, double wind, int ntracer, int nlayer, const double *h,
                       const double *d, const double *salt, const double *temp, const double *y,
                       double *ybgc, int nparam, const double *u, int nsub)
{
    (void)t; (void)lat; (void)dayfrac; (void)wind; (void)salt; (void)temp;
    if (nlayer < 1 || nlayer > M3D_MAX_LAYERS || nsub < 1 || !h || !d || !y || !ybgc)
        return fail(nullptr, M3D_ERR_ARG, "metos3d_bgc: bad sizes or null arrays");
    if (model_id == M3D_MODEL_NDOP) {
        if (ntracer != 2 || nparam != 7 || !u) return fail(nullptr, M3D_ERR_ARG, "metos3d_bgc: PO4-DOP needs 2 tracers, 7 parameters");
    } else if (model_id == M3D_MODEL_NONE) {
        if (ntracer < 1 || ntracer > M3D_MAX_TRACERS) return fail(nullptr, M3D_ERR_ARG, "metos3d_bgc: bad tracer count");
    } else {
        return fail(nullptr, M3D_ERR_UNSUPPORTED, "metos3d_bgc: unknown model %d", model_id);
    }
    size_t ny = (size_t)ntracer * nlayer;
    double *buf = nullptr;
    size_t tot = 2 * (size_t)nlayer + 2 * ny + 8;
    if (cudaMalloc((void **)&buf, sizeof(double) * tot) != cudaSuccess)
        return fail(nullptr, M3D_ERR_CUDA, "metos3d_bgc: cudaMalloc failed");
    double *dh = buf, *dd = buf + nlayer, *dy = buf + 2 * nlayer, *dyb = dy + ny, *du = dyb + ny;
    cudaError_t e = cudaMemcpy(dh, h, sizeof(double) * nlayer, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dd, d, sizeof(double) * nlayer, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dy, y, sizeof(double) * ny, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && model_id == M3D_MODEL_NDOP) e = cudaMemcpy(du, u, sizeof(double) * 7, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        if (model_id == M3D_MODEL_NONE) e = cudaMemset(dyb, 0, sizeof(double) * ny);
        else {
            k_bgc_column<<<1, M3D_MAX_LAYERS>>>(model_id, dt, insol, ice, nlayer, dh, dd, dy, dyb, du, nsub);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaMemcpy(ybgc, dyb, sizeof(double) * ny, cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return fail(nullptr, M3D_ERR_CUDA, "metos3d_bgc: %s", cudaGetErrorString(e));
    return M3D_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------ internal
m3d_status m3d_set_params(m3d_ctx *c, const double *u, cudaMemcpyKind kind)
{
    if (c->nparam > 0)
        CUDA_OR_FAIL(c, cudaMemcpyAsync(c->u_dev, u, sizeof(double) * c->nparam, kind, c->stream));
    return M3D_OK;
}

m3d_status m3d_year_device(m3d_ctx *c, const double *y0, double *y1)
{
    if (c->ens) return ens_run(c, 0, -1, y0, y1);
    size_t len = sizeof(double) * (size_t)c->ntr * c->n;
    if (c->plan == M3D_PLAN_GRAPH && !c->year_graph) {
        m3d_status st = build_year_graph(c);
        if (st != M3D_OK) return st;
    }
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->ybuf[0], y0, len, cudaMemcpyDeviceToDevice, c->stream));
    return run_year_from_ybuf(c, y1, cudaMemcpyDeviceToDevice);
}

cudaError_t m3d_alloc(m3d_ctx *c, void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 1);
    if (e == cudaSuccess) c->allocs.push_back(*p);
    return e;
}

m3d_status m3d_year_record_device(m3d_ctx *c, const double *y0, double *y1, double *fn)
{
    if (!c->lin_ok && !c->lin_tri_ok) return fail(c, M3D_ERR_UNSUPPORTED, "this context has no linearised year map");
    if (c->plan != M3D_PLAN_RESIDENT) return fail(c, M3D_ERR_UNSUPPORTED, "recording needs the resident plan");
    double *saved = c->P.fn_out;
    c->P.fn_out = fn;
    m3d_status st = m3d_year_device(c, y0, y1);
    c->P.fn_out = saved;
    return st;
}

m3d_status m3d_year_linear_device(m3d_ctx *c, const double *fn, const double *v, double *jv)
{
    const size_t len = sizeof(double) * (size_t)c->ntr * c->n;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->ybuf[0], v, len, cudaMemcpyDeviceToDevice, c->stream));
    return run_year_linear(c, fn, jv);
}

m3d_status m3d_year_tangent_device(m3d_ctx *c, const double *y0, const double *v, double *phi, double *jv)
{
    if (c->tangent_form == M3D_TANGENT_LINEARISED) {
        if (!c->fn_buf) {
            void *p = nullptr;
            CUDA_OR_FAIL(c, m3d_alloc(c, &p, sizeof(double) * (size_t)c->nstep * (size_t)std::max(c->P.n_eu, 1)));
            c->fn_buf = (double *)p;
        }
        m3d_status st = m3d_year_record_device(c, y0, phi, c->fn_buf);
        if (st != M3D_OK) return st;
        return m3d_year_linear_device(c, c->fn_buf, v, jv);
    }
    if (c->ens_tan) return ens_tangent_run(c, y0, v, phi, jv);
    if (!c->tan_ok) return fail(c, M3D_ERR_UNSUPPORTED, "this model has no tangent year kernel");
    const size_t half = sizeof(double) * (size_t)c->ntr * c->n;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->ybuf[0], y0, half, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_OR_FAIL(c, cudaMemcpyAsync((char *)c->ybuf[0] + half, v, half, cudaMemcpyDeviceToDevice, c->stream));
    return run_year_tangent(c, phi, jv);
}

extern "C" m3d_status metos3d_year_tangent(m3d_ctx *c, const double *y0, const double *v, const double *u,
                                           double *phi_out, double *jv_out)
{
    if (!c) return fail(nullptr, M3D_ERR_ARG, "metos3d_year_tangent: null context");
    if (!y0 || !v || !phi_out || !jv_out || (c->nparam > 0 && !u))
        return fail(c, M3D_ERR_ARG, "metos3d_year_tangent: null pointer");
    m3d_status st = m3d_set_params(c, u, cudaMemcpyDeviceToDevice);
    if (st != M3D_OK) return st;
    return m3d_year_tangent_device(c, y0, v, phi_out, jv_out);
}

m3d_status m3d_prologue(m3d_ctx *c) { return launch_prologue(c, c->u_dev); }

m3d_status m3d_ens_sync_params(m3d_ctx *c) { return ens_sync_params(c); }

m3d_status m3d_step_device(m3d_ctx *c, int j, const double *y, double *yn) { return launch_step(c, j, y, yn); }
