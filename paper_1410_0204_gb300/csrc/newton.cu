// newton.cu -- spin-up and the matrix-free Newton-Krylov periodic solve (Metos3D,
// arXiv:1410.0204, Sections 4, 6 and 7) on the device.
//
// F(y) = y - phi(y) = 0 is solved by Newton's method, globalised by a backtracking line
// search with cubic interpolation; each Newton system (I - phi'(y)) s = -F(y) is solved
// inexactly by restarted GMRES with modified Gram-Schmidt orthogonalisation, with the
// inner tolerances of Eisenstat and Walker.  The Jacobian-vector products are finite
// differences of the year map.  All vectors stay on the device; the Gram-Schmidt
// coefficients are computed and applied on the device, and the host reads one column of
// the Hessenberg matrix per Krylov iteration to update its Givens rotations.
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

struct Workspace {
    int m = 0;
    long long N = 0;
    double *V = nullptr;        // [m+1][N] Krylov basis
    double *w = nullptr, *F = nullptr, *py = nullptr, *s = nullptr, *y = nullptr;
    double *yn = nullptr, *pyn = nullptr, *tmp = nullptr, *phv = nullptr, *x = nullptr;
    double *H = nullptr;        // [m+1][m] column-major Hessenberg (device)
    double *part = nullptr, *scal = nullptr;
};

struct Solver {
    m3d_ctx *c;
    Workspace W;
    long long N;
    int grid;
    bool tangent = false;           // Jacobian-vector products by the tangent year map
    int *tangent_maps = nullptr;

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
    if (S.tangent) {
        (*S.tangent_maps)++;
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

// Restarted GMRES(m) with modified Gram-Schmidt for A x = b, x0 = 0.  res_rel (may be null)
// receives the last residual estimate relative to ||b||.
m3d_status gmres(Solver &S, const Operator &apply, const double *b, double *x, double tol_rel, int maxit, int *iters,
                 double *res_rel = nullptr)
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
    if (res_rel) *res_rel = 0.0;
    if (bnorm == 0.0) return M3D_OK;
    double *r = W.w;                               // the first residual is b itself
    double beta = bnorm;
    st = S.axpby(W.V, 1.0 / beta, b, 0.0, b);
    if (st != M3D_OK) return st;
    std::vector<double> Hh((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), col(m + 1), yk(m);
    while (true) {
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int k_used = 0;
        bool done = false;
        for (int k = 0; k < m; k++) {
            double *vk = W.V + (size_t)k * N;
            double *hk = W.H + (size_t)k * (m + 1);
            st = apply(vk, 1.0, W.w);
            if (st != M3D_OK) return st;
            for (int i = 0; i <= k; i++) {            // modified Gram-Schmidt, coefficients on the device
                const double *vi = W.V + (size_t)i * N;
                st = S.dot_dev(W.w, vi, hk + i, false);
                if (st != M3D_OK) return st;
                k_sub_scaled<<<S.grid, 256, 0, c->stream>>>(W.w, vi, hk + i, N);
                st = S.launch_ok();
                if (st != M3D_OK) return st;
            }
            st = S.dot_dev(W.w, W.w, hk + k + 1, true);
            if (st != M3D_OK) return st;
            st = S.read(hk, col.data(), k + 2);
            if (st != M3D_OK) return st;
            if (col[k + 1] > 0.0) {
                st = S.axpby(W.V + (size_t)(k + 1) * N, 1.0 / col[k + 1], W.w, 0.0, W.w);
                if (st != M3D_OK) return st;
            }
            for (int i = 0; i < k; i++) {             // previous Givens rotations
                double t = cs[i] * col[i] + sn[i] * col[i + 1];
                col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
                col[i] = t;
            }
            double d = std::hypot(col[k], col[k + 1]);
            if (d == 0.0) { cs[k] = 1.0; sn[k] = 0.0; }
            else { cs[k] = col[k] / d; sn[k] = col[k + 1] / d; }
            col[k] = d;
            col[k + 1] = 0.0;
            for (int i = 0; i <= k; i++) Hh[(size_t)k * (m + 1) + i] = col[i];
            g[k + 1] = -sn[k] * g[k];
            g[k] = cs[k] * g[k];
            (*iters)++;
            k_used = k + 1;
            if (std::fabs(g[k + 1]) <= tol_rel * bnorm || *iters >= maxit || d == 0.0) {
                done = std::fabs(g[k + 1]) <= tol_rel * bnorm || *iters >= maxit || d == 0.0;
                break;
            }
        }
        // back substitution for the upper triangular least-squares system, then x += V y
        for (int i = k_used - 1; i >= 0; i--) {
            double s = g[i];
            for (int j = i + 1; j < k_used; j++) s -= Hh[(size_t)j * (m + 1) + i] * yk[j];
            double dii = Hh[(size_t)i * (m + 1) + i];
            yk[i] = dii != 0.0 ? s / dii : 0.0;
        }
        for (int i = 0; i < k_used; i++) {
            st = S.axpby(x, 1.0, x, yk[i], W.V + (size_t)i * N);
            if (st != M3D_OK) return st;
        }
        if (res_rel) *res_rel = std::fabs(g[k_used]) / bnorm;
        if (done && (std::fabs(g[k_used]) <= tol_rel * bnorm || *iters >= maxit)) break;
        // restart from the true residual r = b - J x
        double xnorm = 0.0;
        st = S.norm(x, &xnorm);
        if (st != M3D_OK) return st;
        st = apply(x, xnorm, W.tmp);
        if (st != M3D_OK) return st;
        st = S.axpby(r, 1.0, b, -1.0, W.tmp);
        if (st != M3D_OK) return st;
        st = S.norm(r, &beta);
        if (st != M3D_OK) return st;
        if (res_rel) *res_rel = beta / bnorm;
        if (beta <= tol_rel * bnorm || *iters >= maxit) break;
        st = S.axpby(W.V, 1.0 / beta, r, 0.0, r);
        if (st != M3D_OK) return st;
    }
    return M3D_OK;
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
    return M3D_OK;
}

// Release a workspace allocated through m3d_alloc (it is also freed with the context).
void release_workspace(m3d_ctx *c, Workspace &W)
{
    void *ptrs[] = {W.V, W.w, W.F, W.py, W.s, W.y, W.yn, W.pyn, W.tmp, W.phv, W.x, W.H, W.part, W.scal};
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
    S.tangent_maps = &R.tangent_maps;
    m3d_status st = ensure_workspace(c, S, o.restart);
    if (st != M3D_OK) { release_workspace(c, S.W); return st; }
    Workspace &W = S.W;
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
    TRY(S.phi(W.y, W.py, &R.year_maps));
    TRY(metos3d_sync(c));
    TRY(S.axpby(W.F, 1.0, W.y, -1.0, W.py));
    double r = 0.0;
    TRY(S.norm(W.F, &r));
    R.residual0 = r;
    R.residuals[0] = r;
    const double gamma = 0.9, alpha = 0.5 * (1.0 + std::sqrt(5.0));
    double eta_prev = -1.0, r_prev = 0.0;
    while (R.newton_steps < o.max_newton && r > o.tol) {
        double eta;
        if (eta_prev < 0.0) eta = 0.3;
        else {
            eta = gamma * std::pow(r / r_prev, alpha);
            double safe = gamma * std::pow(eta_prev, alpha);
            if (safe > 0.1) eta = std::max(eta, safe);
        }
        eta = std::min(std::max(eta, 0.5 * o.tol / r), 0.9);
        double ynorm = 0.0;
        TRY(S.norm(W.y, &ynorm));
        TRY(S.axpby(W.tmp, -1.0, W.F, 0.0, W.F));                 // b = -F (tmp is reused inside gmres)
        TRY(S.axpby(W.yn, 1.0, W.tmp, 0.0, W.tmp));               // keep b in yn during the solve
        int its = 0;
        const Operator jac = [&](const double *v, double vnorm, double *w) {
            return apply_jacobian(S, W.y, W.py, ynorm, o.fd_eps, v, vnorm, w, &R.year_maps);
        };
        TRY(gmres(S, jac, W.yn, W.s, eta, o.max_krylov, &its));
        R.krylov_total += its;
        // project the step onto zero-mass directions: s -= (w.s / w.w) w
        double ms = 0.0;
        TRY(S.mass(W.s, &ms));
        k_sub_mass<<<S.grid, 256, 0, c->stream>>>(W.s, c->vol, c->n, ms / wsum, N);
        TRY(S.launch_ok());
        R.krylov[std::min(R.newton_steps, M3D_NEWTON_MAX_HIST - 1)] = its;
        // line search on f = |F|^2 / 2 along s
        double f0 = 0.5 * r * r, slope = -r * r, lam = 1.0, lam_prev = -1.0, f_prev = 0.0, fn = 0.0;
        while (true) {
            TRY(S.axpby(W.yn, 1.0, W.y, lam, W.s));
            TRY(S.phi(W.yn, W.pyn, &R.year_maps));
            TRY(metos3d_sync(c));
            TRY(S.axpby(W.tmp, 1.0, W.yn, -1.0, W.pyn));
            double rn = 0.0;
            TRY(S.norm(W.tmp, &rn));
            fn = 0.5 * rn * rn;
            if (!o.line_search || fn <= f0 + 1e-4 * lam * slope || lam < 1e-4) break;
            double lt;
            if (lam_prev < 0.0) lt = -slope / (2.0 * (fn - f0 - slope));
            else {
                double a1 = fn - f0 - lam * slope, a2 = f_prev - f0 - lam_prev * slope, den = lam - lam_prev;
                double a = (a1 / (lam * lam) - a2 / (lam_prev * lam_prev)) / den;
                double b = (-lam_prev * a1 / (lam * lam) + lam * a2 / (lam_prev * lam_prev)) / den;
                if (a == 0.0) lt = -slope / (2.0 * b);
                else lt = (-b + std::sqrt(std::max(b * b - 3.0 * a * slope, 0.0))) / (3.0 * a);
            }
            lam_prev = lam;
            f_prev = fn;
            lam = std::min(std::max(lt, 0.1 * lam), 0.5 * lam);
        }
        std::swap(W.y, W.yn);
        std::swap(W.py, W.pyn);
        std::swap(W.F, W.tmp);
        r_prev = r;
        eta_prev = eta;
        r = std::sqrt(2.0 * fn);
        R.newton_steps++;
        R.residuals[std::min(R.newton_steps, M3D_NEWTON_MAX_HIST - 1)] = r;
        R.lambdas[std::min(R.newton_steps - 1, M3D_NEWTON_MAX_HIST - 1)] = lam;
    }
#undef TRY
    R.residual = r;
    R.converged = r <= o.tol;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(y_io, W.y, sizeof(double) * N, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    m3d_status out = R.converged ? M3D_OK : M3D_NOT_CONVERGED;
    if (!R.converged) fail(c, M3D_NOT_CONVERGED, "Newton stopped at residual %.3e after %d steps", r, R.newton_steps);
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
    TRY(gmres(S, adjoint_op, W.F, W.x, o.tol, o.max_krylov, &its, &est));
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
