// newton.cu -- spin-up and the matrix-free Newton-Krylov periodic solve (Metos3D,
// arXiv:1410.0204, Sections 4, 6 and 7) on the device.
//
// F(y) = y - phi(y) = 0 is solved by Newton's method, globalised by a backtracking line
// search with cubic interpolation; each Newton system (I - phi'(y)) s = -F(y) is solved
// inexactly by restarted GMRES with modified Gram-Schmidt orthogonalisation, with the
// inner tolerances of Eisenstat and Walker.  The Jacobian-vector products are finite
// differences of the year map or the tangent year map.  All vectors stay on the device, and
// so does the Krylov loop: the Gram-Schmidt coefficients, the Givens rotations of the
// Hessenberg matrix and the convergence test are kernels, and the host reads a small status
// record per iteration one iteration late, while the next one is already queued.
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <vector>

#include "context.h"

namespace {

constexpr int kRedBlocks = 256;
constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_reduce(double v, double *ws)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += ws[i];
    return s;
}

// part[block] = sum over the block's grid-stride share of a[i] * b[i]
__global__ void __launch_bounds__(kRedThreads) k_dot_part(const double *a, const double *b, long long len,
                                                          double *part)
{
    __shared__ double ws[kRedThreads / 32];
    double v = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
        v += a[i] * b[i];
    double s = block_reduce(v, ws);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// part[block] = sum over the block's share of vol[i mod n] * a[i] (the mass of a)
__global__ void __launch_bounds__(kRedThreads) k_mass_part(const double *a, const double *vol, int n, long long len,
                                                           double *part)
{
    __shared__ double ws[kRedThreads / 32];
    double v = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
        v += vol[i % n] * a[i];
    double s = block_reduce(v, ws);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out[0] = sum of part (fixed order), or its square root
__global__ void k_finish(const double *part, int np, double *out, int take_sqrt)
{
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < np; i++) s += part[i];
        out[0] = take_sqrt ? sqrt(s) : s;
    }
}

// y -= coef[0] * x
__global__ void k_sub_scaled(double *y, const double *x, const double *coef, long long len)
{
    const double c = coef[0];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
        y[i] = fma(-c, x[i], y[i]);
}

// z = a x + b y
__global__ void k_axpby(double *z, double a, const double *x, double b, const double *y, long long len)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
        z[i] = a * x[i] + b * y[i];
}

// w = v - (phv - py) / h
__global__ void k_fd_jv(double *w, const double *v, const double *phv, const double *py, double h, long long len)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
        w[i] = v[i] - (phv[i] - py[i]) / h;
}

// s -= c vol[i mod n]
__global__ void k_sub_mass(double *s, const double *vol, int n, double c, long long len)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
        s[i] = fma(-c, vol[i % n], s[i]);
}

// ---- GMRES cycle state on the device.  The host enqueues the Krylov iterations of a cycle
// without reading anything back: the Hessenberg column, its Givens rotation and the
// convergence test are all evaluated by kernels, and the host learns the outcome of
// iteration k only while iteration k+1 is already queued (a pinned copy of this struct
// behind an event).  Once `done` is set, the year-map kernels of the iterations still in the
// queue return at once (SyncParams::skip) and the Givens kernel ignores them.
struct KrylovStatus {
    int done;                   // converged, broken down, or out of iterations
    int k_used;                 // Krylov vectors of the cycle's solution
    int iters;                  // iterations over all cycles of the solve
    int maxit;
    double tol_abs;             // tol_rel ||b||
    double res;                 // |g[k_used]|, the cycle's residual norm estimate
};

struct Workspace {
    int m = 0;
    long long N = 0;
    double *V = nullptr;        // [m+1][N] Krylov basis
    double *w = nullptr, *F = nullptr, *py = nullptr, *s = nullptr, *y = nullptr;
    double *yn = nullptr, *pyn = nullptr, *tmp = nullptr, *phv = nullptr, *x = nullptr;
    double *H = nullptr;        // [m+1][m] column-major Hessenberg (device)
    double *part = nullptr, *scal = nullptr;
    double *g = nullptr, *cs = nullptr, *sn = nullptr, *yk = nullptr;   // [m+1], [m], [m], [m] (device)
    double *fn_cur = nullptr, *fn_next = nullptr;   // recorded source-term Jacobians (linearised tangent)
    KrylovStatus *kst = nullptr;              // device
    KrylovStatus *kst_host = nullptr;         // pinned, three slots
    cudaEvent_t ev[2] = {nullptr, nullptr};
};

struct Solver {
    m3d_ctx *c;
    Workspace W;
    long long N;
    int grid;
    bool tangent = false;           // Jacobian-vector products by the tangent year map
    bool linear = false;            // ... by the linearised sweep about the recorded trajectory
    int applies = 0;                // operator applications a GMRES call carried out

    m3d_status launch_ok() { CUDA_OR_FAIL(c, cudaGetLastError()); return M3D_OK; }

    // dot product of two vectors of `len` entries (default: the state length) into the device scalar *out
    m3d_status dot_dev(const double *a, const double *b, double *out, bool take_sqrt, long long len = -1)
    {
        k_dot_part<<<kRedBlocks, kRedThreads, 0, c->stream>>>(a, b, len < 0 ? N : len, W.part);
        k_finish<<<1, 32, 0, c->stream>>>(W.part, kRedBlocks, out, take_sqrt ? 1 : 0);
        return launch_ok();
    }

    // total mass sum_i vol[i mod n] a[i], on the host
    m3d_status mass(const double *a, double *out_host)
    {
        k_mass_part<<<kRedBlocks, kRedThreads, 0, c->stream>>>(a, c->vol, c->n, N, W.part);
        k_finish<<<1, 32, 0, c->stream>>>(W.part, kRedBlocks, W.scal, 0);
        m3d_status st = launch_ok();
        if (st != M3D_OK) return st;
        return read(W.scal, out_host, 1);
    }

    m3d_status read(const double *dev, double *host, int count)
    {
        CUDA_OR_FAIL(c, cudaMemcpyAsync(host, dev, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream));
        CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
        return M3D_OK;
    }

    m3d_status norm(const double *a, double *out_host)
    {
        m3d_status st = dot_dev(a, a, W.scal, true);
        if (st != M3D_OK) return st;
        return read(W.scal, out_host, 1);
    }

    m3d_status axpby(double *z, double a, const double *x, double b, const double *y)
    {
        k_axpby<<<grid, 256, 0, c->stream>>>(z, a, x, b, y, N);
        return launch_ok();
    }

    m3d_status phi(const double *y, double *out, int *count)
    {
        (*count)++;
        return m3d_year_device(c, y, out);
    }
};

// J v = v - phi'(y) v: by the tangent year map, or by finite differences
// v - (phi(y + h v) - phi(y)) / h with h = eps ||y|| / ||v||
m3d_status apply_jacobian(Solver &S, const double *y, const double *py, double ynorm, double eps,
                          const double *v, double vnorm, double *w, int *year_maps)
{
    if (S.linear) {
        m3d_status st = m3d_year_linear_device(S.c, S.W.fn_cur, v, S.W.tmp);
        if (st != M3D_OK) return st;
        k_axpby<<<S.grid, 256, 0, S.c->stream>>>(w, 1.0, v, -1.0, S.W.tmp, S.N);
        return S.launch_ok();
    }
    if (S.tangent) {
        m3d_status st = m3d_year_tangent_device(S.c, y, v, S.W.phv, S.W.tmp);
        if (st != M3D_OK) return st;
        k_axpby<<<S.grid, 256, 0, S.c->stream>>>(w, 1.0, v, -1.0, S.W.tmp, S.N);
        return S.launch_ok();
    }
    double h = eps * ynorm / vnorm;
    if (!(h > 0.0)) h = eps;
    m3d_status st = S.axpby(S.W.tmp, 1.0, y, h, v);
    if (st != M3D_OK) return st;
    st = S.phi(S.W.tmp, S.W.phv, year_maps);
    if (st != M3D_OK) return st;
    k_fd_jv<<<S.grid, 256, 0, S.c->stream>>>(w, v, S.W.phv, py, h, S.N);
    return S.launch_ok();
}

// w = A v for a vector v of norm vnorm (the operator of a Krylov solve).
using Operator = std::function<m3d_status(const double *v, double vnorm, double *w)>;

// Start a cycle from the residual of norm *beta (device): g = beta e_1.
__global__ void k_krylov_begin(KrylovStatus *st, const double *beta, double *g, int m)
{
    for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = (i == 0) ? beta[0] : 0.0;
    if (threadIdx.x == 0) {
        st->done = 0;
        st->k_used = 0;
        st->res = beta[0];
    }
}

// out = in / den[0] (zero when den[0] is not positive: a breakdown, which ends the cycle)
__global__ void k_scale_inv(double *out, const double *in, const double *den, long long len)
{
    const double d = den[0];
    const double s = d > 0.0 ? 1.0 / d : 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
        out[i] = s * in[i];
}

// Column k of the Hessenberg matrix (h[0..k+1], column-major with leading dimension m+1):
// apply the cycle's previous rotations, form the rotation that zeroes h[k+1], rotate the
// right-hand side g, and decide whether the cycle is done.  One thread.
__global__ void k_givens(double *H, int m, int k, double *cs, double *sn, double *g, KrylovStatus *st)
{
    if (threadIdx.x != 0 || st->done) return;
    double *h = H + (size_t)k * (m + 1);
    for (int i = 0; i < k; i++) {
        const double t = cs[i] * h[i] + sn[i] * h[i + 1];
        h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
        h[i] = t;
    }
    const double d = hypot(h[k], h[k + 1]);
    if (d == 0.0) {
        cs[k] = 1.0;
        sn[k] = 0.0;
    } else {
        cs[k] = h[k] / d;
        sn[k] = h[k + 1] / d;
    }
    h[k] = d;
    h[k + 1] = 0.0;
    g[k + 1] = -sn[k] * g[k];
    g[k] = cs[k] * g[k];
    st->iters += 1;
    st->k_used = k + 1;
    st->res = fabs(g[k + 1]);
    if (st->res <= st->tol_abs || st->iters >= st->maxit || d == 0.0 || k + 1 == m) st->done = 1;
}

// The cycle's correction: back substitution R y = g on the k_used leading columns, then
// x += V y.  One block; the triangular solve on thread 0, the sum over the basis by all.
__global__ void k_krylov_solution(const double *H, int m, const double *g, const KrylovStatus *st, double *yk)
{
    if (threadIdx.x != 0) return;
    const int ku = st->k_used;
    for (int i = ku - 1; i >= 0; i--) {
        double s = g[i];
        for (int j = i + 1; j < ku; j++) s -= H[(size_t)j * (m + 1) + i] * yk[j];
        const double dii = H[(size_t)i * (m + 1) + i];
        yk[i] = dii != 0.0 ? s / dii : 0.0;
    }
}

__global__ void k_add_basis(double *x, const double *V, const double *yk, const KrylovStatus *st, long long N)
{
    const int ku = st->k_used;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        double s = x[i];
        for (int j = 0; j < ku; j++) s = fma(yk[j], V[(size_t)j * N + i], s);
        x[i] = s;
    }
}

// Restarted GMRES(m) with modified Gram-Schmidt for A x = b, x0 = 0, iterations and
// rotations on the device.  res_rel (may be null) receives the last residual estimate
// relative to ||b||.  With lag = 1 the host checks iteration k's status only after it has
// queued iteration k+1 (the operator's year-map kernels must honour SyncParams::skip);
// lag = 0 waits for each iteration's status before queuing the next.
m3d_status gmres(Solver &S, const Operator &apply, const double *b, double *x, double tol_rel, int maxit, int *iters,
                 double *res_rel = nullptr, int lag = 1)
{
    m3d_ctx *c = S.c;
    Workspace &W = S.W;
    const int m = W.m;
    const long long N = S.N;
    CUDA_OR_FAIL(c, cudaMemsetAsync(x, 0, sizeof(double) * N, c->stream));
    double bnorm = 0.0;
    m3d_status st = S.norm(b, &bnorm);
    if (st != M3D_OK) return st;
    *iters = 0;
    S.applies = 0;
    if (res_rel) *res_rel = 0.0;
    if (bnorm == 0.0) return M3D_OK;
    KrylovStatus init{0, 0, 0, maxit, tol_rel * bnorm, bnorm};
    CUDA_OR_FAIL(c, cudaMemcpyAsync(W.kst, &init, sizeof init, cudaMemcpyHostToDevice, c->stream));
    double *r = W.w;                               // the first residual is b itself
    const double *rv = b;
    double *beta_dev = W.scal + 1;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(beta_dev, W.scal, sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    const int *saved_skip = c->S.skip;
    c->S.skip = lag ? &W.kst->done : nullptr;
    auto restore = [&](m3d_status s2) { c->S.skip = saved_skip; return s2; };
    KrylovStatus host{};
    while (true) {
        k_krylov_begin<<<1, 256, 0, c->stream>>>(W.kst, beta_dev, W.g, m);
        k_scale_inv<<<S.grid, 256, 0, c->stream>>>(W.V, rv, beta_dev, N);
        st = S.launch_ok();
        if (st != M3D_OK) return restore(st);
        int queued = 0;
        for (int k = 0; k < m && *iters + queued < maxit; k++) {
            double *vk = W.V + (size_t)k * N;
            double *hk = W.H + (size_t)k * (m + 1);
            st = apply(vk, 1.0, W.w);
            if (st != M3D_OK) return restore(st);
            for (int i = 0; i <= k; i++) {            // modified Gram-Schmidt, coefficients on the device
                const double *vi = W.V + (size_t)i * N;
                st = S.dot_dev(W.w, vi, hk + i, false);
                if (st != M3D_OK) return restore(st);
                k_sub_scaled<<<S.grid, 256, 0, c->stream>>>(W.w, vi, hk + i, N);
            }
            st = S.dot_dev(W.w, W.w, hk + k + 1, true);
            if (st != M3D_OK) return restore(st);
            k_scale_inv<<<S.grid, 256, 0, c->stream>>>(W.V + (size_t)(k + 1) * N, W.w, hk + k + 1, N);
            k_givens<<<1, 32, 0, c->stream>>>(W.H, m, k, W.cs, W.sn, W.g, W.kst);
            st = S.launch_ok();
            if (st != M3D_OK) return restore(st);
            KrylovStatus *slot = W.kst_host + (k & 1);
            CUDA_OR_FAIL(c, cudaMemcpyAsync(slot, W.kst, sizeof(KrylovStatus), cudaMemcpyDeviceToHost, c->stream));
            CUDA_OR_FAIL(c, cudaEventRecord(W.ev[k & 1], c->stream));
            queued++;
            // the outcome of iteration k - lag: the GPU is busy with the iterations queued since
            const int kc = k - lag;
            if (kc >= 0) {
                CUDA_OR_FAIL(c, cudaEventSynchronize(W.ev[kc & 1]));
                if (W.kst_host[kc & 1].done) break;
            }
        }
        CUDA_OR_FAIL(c, cudaMemcpyAsync(W.kst_host + 2, W.kst, sizeof(KrylovStatus), cudaMemcpyDeviceToHost, c->stream));
        k_krylov_solution<<<1, 32, 0, c->stream>>>(W.H, m, W.g, W.kst, W.yk);
        k_add_basis<<<S.grid, 256, 0, c->stream>>>(x, W.V, W.yk, W.kst, N);
        st = S.launch_ok();
        if (st != M3D_OK) return restore(st);
        CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
        host = W.kst_host[2];
        S.applies += host.iters - *iters;
        *iters = host.iters;
        if (res_rel) *res_rel = host.res / bnorm;
        if (host.res <= tol_rel * bnorm || *iters >= maxit) break;
        // restart from the true residual r = b - A x
        double xnorm = 0.0;
        st = S.norm(x, &xnorm);
        if (st != M3D_OK) return restore(st);
        c->S.skip = nullptr;
        S.applies++;
        st = apply(x, xnorm, W.tmp);
        c->S.skip = lag ? &W.kst->done : nullptr;
        if (st != M3D_OK) return restore(st);
        st = S.axpby(r, 1.0, b, -1.0, W.tmp);
        if (st != M3D_OK) return restore(st);
        double beta = 0.0;
        st = S.dot_dev(r, r, beta_dev, true);
        if (st != M3D_OK) return restore(st);
        st = S.read(beta_dev, &beta, 1);
        if (st != M3D_OK) return restore(st);
        if (res_rel) *res_rel = beta / bnorm;
        if (beta <= tol_rel * bnorm || beta == 0.0) break;
        rv = r;
    }
    return restore(M3D_OK);
}

// Inner tolerance of Newton step k (Eisenstat and Walker, choice 2): 0.3 for the first step,
// then 0.9 (|F_k| / |F_{k-1}|)^((1 + sqrt 5)/2), raised to the safeguard 0.9 eta_{k-1}^((1 + sqrt 5)/2)
// when that exceeds 0.1, and kept within [0.5 tol / |F_k|, 0.9].
double forcing_term(bool first, double r, double r_prev, double eta_prev, double tol)
{
    const double gamma = 0.9, alpha = 0.5 * (1.0 + std::sqrt(5.0));
    double eta = 0.3;
    if (!first) {
        eta = gamma * std::pow(r / r_prev, alpha);
        const double safe = gamma * std::pow(eta_prev, alpha);
        if (safe > 0.1) eta = std::max(eta, safe);
    }
    return std::min(std::max(eta, 0.5 * tol / r), 0.9);
}

// First backtrack: the minimiser of the quadratic q(x) = f0 + slope x + c x^2 with q(lam) = f_lam.
double quadratic_backtrack(double f0, double slope, double lam, double f_lam)
{
    return -slope * lam * lam / (2.0 * (f_lam - f0 - slope * lam));
}

// Later backtracks: the local minimiser of the cubic m(x) = f0 + slope x + b x^2 + a x^3 through
// the last two trials (lam, f_lam) and (lam_prev, f_prev); the quadratic's when a = 0.
double cubic_backtrack(double f0, double slope, double lam, double f_lam, double lam_prev, double f_prev)
{
    const double r1 = f_lam - f0 - lam * slope, r2 = f_prev - f0 - lam_prev * slope;
    const double den = lam - lam_prev;
    const double a = (r1 / (lam * lam) - r2 / (lam_prev * lam_prev)) / den;
    const double b = (-lam_prev * r1 / (lam * lam) + lam * r2 / (lam_prev * lam_prev)) / den;
    if (a == 0.0) return -slope / (2.0 * b);
    return (-b + std::sqrt(std::max(b * b - 3.0 * a * slope, 0.0))) / (3.0 * a);
}

m3d_status ensure_workspace(m3d_ctx *c, Solver &S, int m)
{
    S.N = (long long)c->ntr * c->n;
    S.grid = (int)std::min<long long>((S.N + 255) / 256, 4096);
    Workspace &W = S.W;
    W.m = m;
    W.N = S.N;
    size_t vec = sizeof(double) * (size_t)S.N;
    void *p = nullptr;
    CUDA_OR_FAIL(c, m3d_alloc(c, &p, vec * (size_t)(m + 1)));
    W.V = (double *)p;
    double **vs[] = {&W.w, &W.F, &W.py, &W.s, &W.y, &W.yn, &W.pyn, &W.tmp, &W.phv, &W.x};
    for (double **q : vs) {
        CUDA_OR_FAIL(c, m3d_alloc(c, &p, vec));
        *q = (double *)p;
    }
    CUDA_OR_FAIL(c, m3d_alloc(c, &p, sizeof(double) * (size_t)(m + 1) * m));
    W.H = (double *)p;
    CUDA_OR_FAIL(c, m3d_alloc(c, &p, sizeof(double) * kRedBlocks));
    W.part = (double *)p;
    CUDA_OR_FAIL(c, m3d_alloc(c, &p, sizeof(double) * 4));
    W.scal = (double *)p;
    CUDA_OR_FAIL(c, m3d_alloc(c, &p, sizeof(double) * (size_t)(4 * m + 1)));
    W.g = (double *)p;
    W.cs = W.g + (m + 1);
    W.sn = W.cs + m;
    W.yk = W.sn + m;
    CUDA_OR_FAIL(c, m3d_alloc(c, &p, sizeof(KrylovStatus)));
    W.kst = (KrylovStatus *)p;
    CUDA_OR_FAIL(c, cudaMallocHost(&p, 3 * sizeof(KrylovStatus)));
    W.kst_host = (KrylovStatus *)p;
    for (int i = 0; i < 2; i++) CUDA_OR_FAIL(c, cudaEventCreateWithFlags(&W.ev[i], cudaEventDisableTiming));
    return M3D_OK;
}

// Release a workspace allocated through m3d_alloc (it is also freed with the context).
void release_workspace(m3d_ctx *c, Workspace &W)
{
    if (W.kst_host) cudaFreeHost(W.kst_host);
    for (cudaEvent_t e : W.ev)
        if (e) cudaEventDestroy(e);
    void *ptrs[] = {W.V, W.w, W.F, W.py, W.s, W.y, W.yn, W.pyn, W.tmp, W.phv, W.x, W.H, W.part, W.scal, W.g, W.kst,
                    W.fn_cur, W.fn_next};
    for (void *p : ptrs) {
        if (!p) continue;
        for (size_t i = 0; i < c->allocs.size(); i++)
            if (c->allocs[i] == p) { c->allocs.erase(c->allocs.begin() + i); break; }
        cudaFree(p);
    }
    W = Workspace{};
}

}  // namespace

extern "C" {

void metos3d_newton_default_options(m3d_newton_opts *o)
{
    if (!o) return;
    o->tol = 1e-8;
    o->max_newton = 40;
    o->restart = 200;
    o->max_krylov = 200;
    o->jv = M3D_JV_FD;
    o->fd_eps = 1e-8;
    o->line_search = 1;
}

m3d_status metos3d_spinup(m3d_ctx *c, double *y, const double *u, int nyears, double tol, double *res_host,
                          int *years_done)
{
    if (!c) return fail(nullptr, M3D_ERR_ARG, "metos3d_spinup: null context");
    if (!y || nyears < 0 || (c->nparam > 0 && !u)) return fail(c, M3D_ERR_ARG, "metos3d_spinup: bad arguments");
    Solver S{c, {}, 0, 0};
    S.N = (long long)c->ntr * c->n;
    S.grid = (int)std::min<long long>((S.N + 255) / 256, 4096);
    Workspace &W = S.W;
    void *p = nullptr;
    double **bufs[] = {&W.py, &W.tmp};
    for (double **q : bufs) {
        CUDA_OR_FAIL(c, m3d_alloc(c, &p, sizeof(double) * (size_t)S.N));
        *q = (double *)p;
    }
    CUDA_OR_FAIL(c, m3d_alloc(c, &p, sizeof(double) * kRedBlocks));
    W.part = (double *)p;
    CUDA_OR_FAIL(c, m3d_alloc(c, &p, sizeof(double) * 4));
    W.scal = (double *)p;
    m3d_status st = m3d_set_params(c, u, cudaMemcpyDeviceToDevice);
    int done = 0, maps = 0;
    for (int k = 0; k < nyears && st == M3D_OK; k++) {
        st = S.phi(y, W.py, &maps);                          // phi(y)
        if (st == M3D_OK) st = metos3d_sync(c);
        if (st == M3D_OK) st = S.axpby(W.tmp, 1.0, W.py, -1.0, y);
        double r = 0.0;
        if (st == M3D_OK) st = S.norm(W.tmp, &r);          // ||phi(y) - y||
        if (st != M3D_OK) break;
        cudaError_t e = cudaMemcpyAsync(y, W.py, sizeof(double) * (size_t)S.N, cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) { st = fail(c, M3D_ERR_CUDA, "metos3d_spinup: %s", cudaGetErrorString(e)); break; }
        if (res_host) res_host[k] = r;
        done = k + 1;
        if (r <= tol) break;
    }
    cudaStreamSynchronize(c->stream);
    release_workspace(c, W);
    if (years_done) *years_done = done;
    return st;
}

m3d_status metos3d_newton_solve(m3d_ctx *c, double *y_io, const double *u, const m3d_newton_opts *opts_in,
                                m3d_newton_report *rep)
{
    if (!c) return fail(nullptr, M3D_ERR_ARG, "metos3d_newton_solve: null context");
    if (!y_io || (c->nparam > 0 && !u)) return fail(c, M3D_ERR_ARG, "metos3d_newton_solve: null pointer");
    m3d_newton_opts o;
    metos3d_newton_default_options(&o);
    if (opts_in) o = *opts_in;
    if (!(o.tol > 0.0) || o.max_newton < 0 || o.restart < 1 || o.max_krylov < 1 || !(o.fd_eps > 0.0))
        return fail(c, M3D_ERR_ARG, "metos3d_newton_solve: bad options");
    if (o.jv != M3D_JV_FD && o.jv != M3D_JV_TANGENT) return fail(c, M3D_ERR_ARG, "metos3d_newton_solve: bad jv");
    if (o.jv == M3D_JV_TANGENT && !c->tan_ok)
        return fail(c, M3D_ERR_UNSUPPORTED, "metos3d_newton_solve: this model has no tangent year map");
    auto t0 = std::chrono::steady_clock::now();
    m3d_newton_report R;
    memset(&R, 0, sizeof R);
    Solver S{c, {}, 0, 0};
    S.tangent = o.jv == M3D_JV_TANGENT;
    // exact products by the linearised sweep where the context has it: the line search records
    // the source term's Jacobian along the year maps it evaluates anyway
    S.linear = S.tangent && c->plan == M3D_PLAN_RESIDENT && (c->lin_ok || c->lin_tri_ok);
    m3d_status st = ensure_workspace(c, S, o.restart);
    if (st == M3D_OK && S.linear) {
        void *p = nullptr;
        const size_t fnb = sizeof(double) * (size_t)c->nstep * (size_t)std::max(c->P.n_eu, 1);
        cudaError_t e = m3d_alloc(c, &p, fnb);
        if (e == cudaSuccess) { S.W.fn_cur = (double *)p; e = m3d_alloc(c, &p, fnb); }
        if (e == cudaSuccess) S.W.fn_next = (double *)p;
        if (e != cudaSuccess) st = fail(c, M3D_ERR_CUDA, "metos3d_newton_solve: %s", cudaGetErrorString(e));
    }
    if (st != M3D_OK) { release_workspace(c, S.W); return st; }
    Workspace &W = S.W;
    // phi(y), recording the source term's Jacobian into fn when the products are linearised sweeps
    auto phi_rec = [&](const double *yy, double *out, double *fn) -> m3d_status {
        if (!S.linear) return S.phi(yy, out, &R.year_maps);
        R.year_maps++;
        return m3d_year_record_device(c, yy, out, fn);
    };
    const long long N = S.N;
    auto finish = [&](m3d_status s) {
        R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (rep) *rep = R;
        release_workspace(c, W);
        return s;
    };
#define TRY(x) do { st = (x); if (st != M3D_OK) return finish(st); } while (0)
    TRY(m3d_set_params(c, u, cudaMemcpyDeviceToDevice));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(W.y, y_io, sizeof(double) * N, cudaMemcpyDeviceToDevice, c->stream));
    // zero-mass projection: w = vol repeated per tracer, w.w = ntr sum vol^2
    double wsum = 0.0;
    TRY(S.dot_dev(c->vol, c->vol, W.scal, false, c->n));
    TRY(S.read(W.scal, &wsum, 1));
    wsum *= c->ntr;
    TRY(phi_rec(W.y, W.py, W.fn_cur));
    TRY(metos3d_sync(c));
    TRY(S.axpby(W.F, 1.0, W.y, -1.0, W.py));
    double r = 0.0;
    TRY(S.norm(W.F, &r));
    R.residual0 = r;
    R.residuals[0] = r;
    double eta_prev = 0.0, r_prev = 0.0;
    // the ensemble-backed models run their year as a graph of step launches, which does not
    // honour SyncParams::skip: their Krylov iterations are checked one at a time
    const int lag = c->ens ? 0 : 1;
    while (R.newton_steps < o.max_newton && r > o.tol && std::isfinite(r)) {
        const int step = R.newton_steps, hs = std::min(step, M3D_NEWTON_MAX_HIST - 1);
        const double eta = forcing_term(step == 0, r, r_prev, eta_prev, o.tol);
        double ynorm = 0.0;
        TRY(S.norm(W.y, &ynorm));
        TRY(S.axpby(W.tmp, -1.0, W.F, 0.0, W.F));                 // b = -F (tmp is reused inside gmres)
        TRY(S.axpby(W.yn, 1.0, W.tmp, 0.0, W.tmp));               // keep b in yn during the solve
        int its = 0, fd_maps = 0;
        double res_rel = 0.0;
        const Operator jac = [&](const double *v, double vnorm, double *w) {
            return apply_jacobian(S, W.y, W.py, ynorm, o.fd_eps, v, vnorm, w, &fd_maps);
        };
        TRY(gmres(S, jac, W.yn, W.s, eta, o.max_krylov, &its, &res_rel, lag));
        R.krylov_total += its;
        if (S.tangent) R.tangent_maps += S.applies;
        else R.year_maps += S.applies;
        // project the step onto zero-mass directions: s -= (w.s / w.w) w
        double ms = 0.0;
        TRY(S.mass(W.s, &ms));
        k_sub_mass<<<S.grid, 256, 0, c->stream>>>(W.s, c->vol, c->n, ms / wsum, N);
        TRY(S.launch_ok());
        R.krylov[hs] = its;
        R.etas[hs] = eta;
        // slope of f = |F|^2 / 2 along s: GMRES leaves a residual rho = |F + J s| orthogonal to
        // J s (its minimal-residual property), so F.J s = -(|F|^2 - rho^2)
        const double rho = res_rel * r;
        const double f0 = 0.5 * r * r, slope = -(r * r - rho * rho);
        R.slopes[hs] = slope;
        // Backtracking (Dennis & Schnabel, Algorithm A6.3.1): a trial whose residual is not
        // finite gives no model, the next one is a tenth of it; no step below 1e-4 is tried,
        // and when the search fails the solve stops at its current iterate.
        double lam = 1.0, lam_prev = -1.0, f_prev = 0.0, fn = 0.0;
        int trials = 0;
        bool failed = false;
        while (true) {
            if (o.line_search && lam < 1e-4) {
                failed = true;
                break;
            }
            TRY(S.axpby(W.yn, 1.0, W.y, lam, W.s));
            TRY(phi_rec(W.yn, W.pyn, W.fn_next));
            TRY(metos3d_sync(c));
            TRY(S.axpby(W.tmp, 1.0, W.yn, -1.0, W.pyn));
            double rn = 0.0;
            TRY(S.norm(W.tmp, &rn));
            fn = 0.5 * rn * rn;
            trials++;
            if (R.ntrial < M3D_NEWTON_MAX_TRIALS) R.trial_lambdas[R.ntrial++] = lam;
            if (!o.line_search) break;
            if (!std::isfinite(fn)) {
                lam_prev = -1.0;
                lam *= 0.1;
                continue;
            }
            if (fn <= f0 + 1e-4 * lam * slope) break;
            const double lt = lam_prev < 0.0 ? quadratic_backtrack(f0, slope, lam, fn)
                                             : cubic_backtrack(f0, slope, lam, fn, lam_prev, f_prev);
            lam_prev = lam;
            f_prev = fn;
            lam = std::isfinite(lt) ? std::min(std::max(lt, 0.1 * lam), 0.5 * lam) : 0.1 * lam;
        }
        if (failed) {
            R.newton_steps++;
            R.residuals[std::min(R.newton_steps, M3D_NEWTON_MAX_HIST - 1)] = r;
            R.lambdas[hs] = 0.0;
            R.trials[hs] = trials;
            R.line_search_failed = 1;
            break;
        }
        std::swap(W.y, W.yn);
        std::swap(W.py, W.pyn);
        std::swap(W.F, W.tmp);
        std::swap(W.fn_cur, W.fn_next);
        r_prev = r;
        eta_prev = eta;
        r = std::sqrt(2.0 * fn);
        R.newton_steps++;
        R.residuals[std::min(R.newton_steps, M3D_NEWTON_MAX_HIST - 1)] = r;
        R.lambdas[hs] = lam;
        R.trials[hs] = trials;
    }
#undef TRY
    R.residual = r;
    R.converged = r <= o.tol;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(y_io, W.y, sizeof(double) * N, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    m3d_status out = R.converged ? M3D_OK : M3D_NOT_CONVERGED;
    if (R.line_search_failed)
        fail(c, M3D_NOT_CONVERGED, "Newton stopped at residual %.3e: the line search of step %d found no "
                                   "decrease (step lengths down to 1e-4)", r, R.newton_steps);
    else if (!R.converged)
        fail(c, M3D_NOT_CONVERGED, "Newton stopped at residual %.3e after %d steps", r, R.newton_steps);
    return finish(out);
}

}  // extern "C"

extern "C" {

void metos3d_gradient_default_options(m3d_gradient_opts *o)
{
    if (!o) return;
    o->tol = 1e-8;
    o->restart = 200;
    o->max_krylov = 1000;
    o->ckpt_every = 0;
}

m3d_status metos3d_periodic_gradient(m3d_ctx *c, const double *ystar, const double *u, const double *g,
                                     double *lambda, double *ubar_host, const m3d_gradient_opts *opts,
                                     m3d_gradient_report *rep)
{
    if (!c) return fail(nullptr, M3D_ERR_ARG, "metos3d_periodic_gradient: null context");
    if (!ystar || !u || !g || !ubar_host) return fail(c, M3D_ERR_ARG, "metos3d_periodic_gradient: null pointer");
    m3d_gradient_opts o;
    metos3d_gradient_default_options(&o);
    if (opts) o = *opts;
    if (!(o.tol > 0.0) || o.restart < 1 || o.max_krylov < 1)
        return fail(c, M3D_ERR_ARG, "metos3d_periodic_gradient: bad options");
    auto t0 = std::chrono::steady_clock::now();
    m3d_gradient_report R;
    memset(&R, 0, sizeof R);
    Solver S{c, {}, 0, 0};
    AdjointSweep A;
    m3d_status st = A.begin(c, o.ckpt_every > 0 ? o.ckpt_every : c->nstep);
    if (st != M3D_OK) return st;
    st = ensure_workspace(c, S, o.restart);
    Workspace &W = S.W;
    const long long N = S.N;
    auto finish = [&](m3d_status s) {
        R.reverse_sweeps = A.reverse_sweeps;
        R.forward_years = (double)A.forward_steps / c->nstep;
        R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (rep) *rep = R;
        A.release();
        release_workspace(c, W);
        return s;
    };
    if (st != M3D_OK) return finish(st);
#define TRY(x) do { st = (x); if (st != M3D_OK) return finish(st); } while (0)
    auto cu = [&](cudaError_t e) -> m3d_status {
        return e == cudaSuccess ? M3D_OK : fail(c, M3D_ERR_CUDA, "metos3d_periodic_gradient: %s", cudaGetErrorString(e));
    };
    TRY(A.forward(ystar, u));
    // the zero-mass projection P x = x - (w.x / w.w) w, w = vol repeated per tracer
    double wsum = 0.0;
    TRY(S.dot_dev(c->vol, c->vol, W.scal, false, c->n));
    TRY(S.read(W.scal, &wsum, 1));
    wsum *= c->ntr;
    auto project = [&](double *x) -> m3d_status {
        double m = 0.0;
        m3d_status s2 = S.mass(x, &m);
        if (s2 != M3D_OK) return s2;
        k_sub_mass<<<S.grid, 256, 0, c->stream>>>(x, c->vol, c->n, m / wsum, N);
        return S.launch_ok();
    };
    // w = P (v - phi_y^T v), one reverse sweep
    const Operator adjoint_op = [&](const double *v, double, double *w) -> m3d_status {
        m3d_status s2 = A.reverse(v, W.phv, nullptr);
        if (s2 != M3D_OK) return s2;
        s2 = S.axpby(w, 1.0, v, -1.0, W.phv);
        if (s2 != M3D_OK) return s2;
        return project(w);
    };
    // b = P g; what is left of a g along the mass direction alone is rounding (no gradient at
    // fixed mass), so b is taken as zero when it is that small
    TRY(cu(cudaMemcpyAsync(W.F, g, sizeof(double) * N, cudaMemcpyDeviceToDevice, c->stream)));
    double gnorm = 0.0, bnorm = 0.0;
    TRY(S.norm(W.F, &gnorm));
    TRY(project(W.F));
    TRY(S.norm(W.F, &bnorm));
    if (bnorm <= 1e-13 * gnorm) {
        TRY(cu(cudaMemsetAsync(W.F, 0, sizeof(double) * N, c->stream)));
        bnorm = 0.0;
    }
    int its = 0;
    double est = 0.0;
    TRY(gmres(S, adjoint_op, W.F, W.x, o.tol, o.max_krylov, &its, &est, 0));   // reverse sweeps: no skip
    TRY(project(W.x));
    R.krylov = its;
    // ubar = phi_u^T lambda; the same sweep gives phi_y^T lambda for the true residual
    TRY(A.reverse(W.x, W.phv, ubar_host));
    TRY(S.axpby(W.w, 1.0, W.x, -1.0, W.phv));
    TRY(project(W.w));
    TRY(S.axpby(W.w, 1.0, W.F, -1.0, W.w));
    double rnorm = 0.0;
    TRY(S.norm(W.w, &rnorm));
    R.residual = bnorm > 0.0 ? rnorm / bnorm : 0.0;
    R.converged = est <= o.tol;
    if (lambda) TRY(cu(cudaMemcpyAsync(lambda, W.x, sizeof(double) * N, cudaMemcpyDeviceToDevice, c->stream)));
    TRY(cu(cudaStreamSynchronize(c->stream)));
    c->last_launches = (int)std::min<long long>(A.launches, 1LL << 30);
#undef TRY
    return finish(R.converged ? M3D_OK : M3D_NOT_CONVERGED);
}

}  // extern "C"
