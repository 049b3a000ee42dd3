// ensemble_newton.cu -- the periodic solve of Sections 4, 6 and 7 for every member of an
// ensemble at once: Newton's method on F_m(y_m) = y_m - phi_m(y_m) for each member m, with
// its own inexact GMRES(MGS) solve, Eisenstat-Walker tolerance and backtracking line search,
// the members advancing in lockstep.  Every Krylov iteration takes the Jacobian-vector
// products of all members from ONE launch sequence: the tangent ensemble's year map of the
// members' states and Krylov vectors (exact products, Section 6), or one ensemble year map at
// y + h v (finite differences).  Every line-search trial is one ensemble year map.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "metos3d.h"

namespace {

// out[m] = sum over member m's entries [off[m] n, off[m+1] n) of a[i] b[i]; one block per
// member, fixed order (deterministic).
__global__ void k_member_dot(const double *a, const double *b, const int *off, int n, double *out)
{
    __shared__ double ws[32];
    const int m = blockIdx.x;
    const long long i0 = (long long)off[m] * n, i1 = (long long)off[m + 1] * n;
    double v = 0.0;
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) v += a[i] * b[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) s += ws[k];
        out[m] = s;
    }
}

// z[i] = a[m(i)] x[i] + b[m(i)] y[i] with per-member coefficients (rows of member m).
__global__ void k_member_axpby(double *z, const double *a, const double *x, const double *b, const double *y,
                               const int *row_member, int n, long long len)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
        const int m = row_member[i / n];
        z[i] = a[m] * x[i] + (b[m] != 0.0 ? b[m] * y[i] : 0.0);
    }
}

// s[i] -= c[m(i)] vol[i mod n]: the projection of each member's step on its zero-mass directions.
__global__ void k_member_sub_mass(double *s, const double *c, const double *vol, const int *row_member, int n,
                                  long long len)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
        s[i] -= c[row_member[i / n]] * vol[i % n];
}

// per-member mass: out[m] = sum over member m's rows of vol[i mod n] a[i]
__global__ void k_member_mass(const double *a, const double *vol, const int *off, int n, double *out)
{
    __shared__ double ws[32];
    const int m = blockIdx.x;
    const long long i0 = (long long)off[m] * n, i1 = (long long)off[m + 1] * n;
    double v = 0.0;
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) v += vol[i % n] * a[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) s += ws[k];
        out[m] = s;
    }
}

double forcing(bool first, double r, double r_prev, double eta_prev, double tol)
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

double quad_bt(double f0, double slope, double lam, double fl)
{
    return -slope * lam * lam / (2.0 * (fl - f0 - slope * lam));
}

double cubic_bt(double f0, double slope, double lam, double fl, double lp, double fp)
{
    const double r1 = fl - f0 - lam * slope, r2 = fp - f0 - lp * slope, den = lam - lp;
    const double a = (r1 / (lam * lam) - r2 / (lp * lp)) / den;
    const double b = (-lp * r1 / (lam * lam) + lam * r2 / (lp * lp)) / den;
    if (a == 0.0) return -slope / (2.0 * b);
    return (-b + std::sqrt(std::max(b * b - 3.0 * a * slope, 0.0))) / (3.0 * a);
}

struct Dev {
    std::vector<void *> p;
    cudaError_t alloc(double **x, size_t count)
    {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, sizeof(double) * std::max<size_t>(count, 1));
        if (e == cudaSuccess) { p.push_back(q); *x = (double *)q; }
        return e;
    }
    ~Dev()
    {
        for (void *q : p) cudaFree(q);
    }
};

}  // namespace

extern "C" m3d_status metos3d_ensemble_newton_solve(m3d_ensemble *ens, m3d_ensemble *ens_tan, double *Y,
                                                    const double *vol_host, const m3d_newton_opts *opts_in,
                                                    m3d_newton_report *reports)
{
    if (!ens || !Y || !vol_host) return M3D_ERR_ARG;
    m3d_newton_opts o;
    metos3d_newton_default_options(&o);
    if (opts_in) o = *opts_in;
    if (!(o.tol > 0.0) || o.max_newton < 0 || o.restart < 1 || o.max_krylov < 1 || !(o.fd_eps > 0.0)) return M3D_ERR_ARG;
    const bool tangent = o.jv == M3D_JV_TANGENT;
    if (tangent && !ens_tan) return M3D_ERR_ARG;
    auto t0 = std::chrono::steady_clock::now();
    int nm = 0, W = 0, n = 0, G = 0;
    m3d_status st = metos3d_ensemble_layout(ens, &nm, &W, &n, &G, nullptr);
    if (st != M3D_OK) return st;
    std::vector<int> off(nm + 1);
    metos3d_ensemble_layout(ens, nullptr, nullptr, nullptr, nullptr, off.data());
    if (tangent) {
        int nm2 = 0, W2 = 0, n2 = 0;
        metos3d_ensemble_layout(ens_tan, &nm2, &W2, &n2, nullptr, nullptr);
        if (nm2 != nm || W2 != 2 * W || n2 != n) return M3D_ERR_ARG;
    }
    const int mk = std::max(1, std::min(o.restart, o.max_krylov));   // one GMRES cycle per Newton step
    const long long len = (long long)W * n;
    const int grid = (int)std::min<long long>((len + 255) / 256, 4096);
    std::vector<int> row_member(W);
    for (int m = 0; m < nm; m++)
        for (int r = off[m]; r < off[m + 1]; r++) row_member[r] = m;
    Dev D;
    double *PY, *F, *S, *w, *tmp, *Yt, *PYt, *V, *pk, *pko, *vol, *sc_a, *sc_b, *dots;
    int *off_d = nullptr, *rm_d = nullptr;
    cudaError_t e = cudaSuccess;
    for (double **q : {&PY, &F, &S, &w, &tmp, &Yt, &PYt})
        if (e == cudaSuccess) e = D.alloc(q, (size_t)len);
    if (e == cudaSuccess) e = D.alloc(&V, (size_t)len * (mk + 1));
    if (e == cudaSuccess) e = D.alloc(&pk, tangent ? 2 * (size_t)len : 1);
    if (e == cudaSuccess) e = D.alloc(&pko, tangent ? 2 * (size_t)len : 1);
    if (e == cudaSuccess) e = D.alloc(&vol, (size_t)n);
    if (e == cudaSuccess) e = D.alloc(&sc_a, (size_t)nm);
    if (e == cudaSuccess) e = D.alloc(&sc_b, (size_t)nm);
    if (e == cudaSuccess) e = D.alloc(&dots, (size_t)nm);
    if (e == cudaSuccess) { void *q; e = cudaMalloc(&q, sizeof(int) * (nm + 1)); if (e == cudaSuccess) { D.p.push_back(q); off_d = (int *)q; } }
    if (e == cudaSuccess) { void *q; e = cudaMalloc(&q, sizeof(int) * W); if (e == cudaSuccess) { D.p.push_back(q); rm_d = (int *)q; } }
    if (e == cudaSuccess) e = cudaMemcpy(off_d, off.data(), sizeof(int) * (nm + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(rm_d, row_member.data(), sizeof(int) * W, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(vol, vol_host, sizeof(double) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return M3D_ERR_CUDA;
    cudaStream_t s0 = nullptr;          // the ensembles' calls run on their own streams; sync all
#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return M3D_ERR_CUDA; } while (0)
#define ST(x) do { m3d_status s_ = (x); if (s_ != M3D_OK) return s_; } while (0)
    auto sync = [&]() { return cudaDeviceSynchronize(); };
    auto host_vec = [&](const std::vector<double> &h, double *d) { return cudaMemcpy(d, h.data(), sizeof(double) * nm, cudaMemcpyHostToDevice); };
    auto member_dots = [&](const double *a, const double *b, std::vector<double> &out) -> cudaError_t {
        k_member_dot<<<nm, 256, 0, s0>>>(a, b, off_d, n, dots);
        out.resize(nm);
        return cudaMemcpy(out.data(), dots, sizeof(double) * nm, cudaMemcpyDeviceToHost);
    };
    auto axpby = [&](double *z, const std::vector<double> &a, const double *x, const std::vector<double> &b,
                     const double *y) -> cudaError_t {
        cudaError_t r = host_vec(a, sc_a);
        if (r == cudaSuccess) r = host_vec(b, sc_b);
        if (r != cudaSuccess) return r;
        k_member_axpby<<<grid, 256, 0, s0>>>(z, sc_a, x, sc_b, y, rm_d, n, len);
        return cudaGetLastError();
    };
    std::vector<m3d_newton_report> R(nm);
    for (auto &r : R) memset(&r, 0, sizeof r);
    int year_maps = 0, tangent_maps = 0;
    auto phi = [&](const double *yin, double *yout) -> m3d_status {
        year_maps++;
        // the ensemble runs on its own stream: the inputs made on this one must be complete
        if (sync() != cudaSuccess) return M3D_ERR_CUDA;
        m3d_status s2 = metos3d_ensemble_year_map(ens, yin, yout);
        if (s2 == M3D_OK && sync() != cudaSuccess) s2 = M3D_ERR_CUDA;
        return s2;
    };
    const std::vector<double> one(nm, 1.0), zero(nm, 0.0), mone(nm, -1.0);
    // phi(Y), F = Y - phi(Y), residuals
    ST(phi(Y, PY));
    CK(axpby(F, one, Y, mone, PY));
    std::vector<double> r(nm), rprev(nm, 0.0), etaprev(nm, 0.0), dv;
    CK(member_dots(F, F, dv));
    for (int m = 0; m < nm; m++) {
        r[m] = std::sqrt(dv[m]);
        R[m].residual0 = r[m];
        R[m].residuals[0] = r[m];
    }
    std::vector<double> wsum(nm, 0.0);
    {
        double vv = 0.0;
        std::vector<double> vh(vol_host, vol_host + n);
        for (double x : vh) vv += x * x;
        for (int m = 0; m < nm; m++) wsum[m] = vv * (off[m + 1] - off[m]);
    }
    std::vector<char> stopped(nm, 0);         // members whose line search found no decrease
    for (int it = 0; it < o.max_newton; it++) {
        std::vector<char> act(nm, 0);
        bool any = false;
        for (int m = 0; m < nm; m++) {
            act[m] = !stopped[m] && r[m] > o.tol && std::isfinite(r[m]) && R[m].newton_steps < o.max_newton;
            any = any || act[m];
        }
        if (!any) break;
        std::vector<double> eta(nm, 0.0), ynorm(nm, 0.0);
        for (int m = 0; m < nm; m++)
            if (act[m]) eta[m] = forcing(R[m].newton_steps == 0, r[m], rprev[m], etaprev[m], o.tol);
        CK(member_dots(Y, Y, dv));
        for (int m = 0; m < nm; m++) ynorm[m] = std::sqrt(dv[m]);
        // ---- GMRES per member, in lockstep: V0 = -F / r
        std::vector<double> a0(nm);
        for (int m = 0; m < nm; m++) a0[m] = act[m] ? -1.0 / r[m] : 0.0;
        CK(axpby(V, a0, F, zero, F));
        std::vector<std::vector<double>> H(nm, std::vector<double>((size_t)(mk + 1) * mk, 0.0));
        std::vector<std::vector<double>> cs(nm, std::vector<double>(mk, 0.0)), sn = cs;
        std::vector<std::vector<double>> gg(nm, std::vector<double>(mk + 1, 0.0));
        std::vector<int> kused(nm, 0);
        std::vector<char> kact = act;
        for (int m = 0; m < nm; m++) gg[m][0] = r[m];
        for (int k = 0; k < mk; k++) {
            bool anyk = false;
            for (int m = 0; m < nm; m++) anyk = anyk || kact[m];
            if (!anyk) break;
            double *vk = V + (size_t)k * len;
            // w = J v_k = v_k - phi'(Y) v_k for every member
            if (tangent) {
                tangent_maps++;
                for (int m = 0; m < nm; m++) {
                    CK(cudaMemcpyAsync(pk + (size_t)off[m] * n, Y + (size_t)off[m] * n,
                                       sizeof(double) * (size_t)(off[m + 1] - off[m]) * n, cudaMemcpyDeviceToDevice, s0));
                    CK(cudaMemcpyAsync(pk + len + (size_t)off[m] * n, vk + (size_t)off[m] * n,
                                       sizeof(double) * (size_t)(off[m + 1] - off[m]) * n, cudaMemcpyDeviceToDevice, s0));
                }
                CK(sync());
                ST(metos3d_ensemble_year_map(ens_tan, pk, pko));
                CK(sync());
                CK(axpby(w, one, vk, mone, pko + len));
            } else {
                std::vector<double> h(nm);
                for (int m = 0; m < nm; m++) h[m] = kact[m] ? o.fd_eps * ynorm[m] : 0.0;
                CK(axpby(tmp, one, Y, h, vk));
                ST(phi(tmp, PYt));
                std::vector<double> ih(nm), mih(nm);
                for (int m = 0; m < nm; m++) { ih[m] = h[m] > 0.0 ? 1.0 / h[m] : 0.0; mih[m] = -ih[m]; }
                CK(axpby(w, mih, PYt, ih, PY));          // -(phi(y+hv) - phi(y)) / h
                CK(axpby(w, one, w, one, vk));
            }
            // modified Gram-Schmidt per member
            for (int i = 0; i <= k; i++) {
                const double *vi = V + (size_t)i * len;
                CK(member_dots(w, vi, dv));
                std::vector<double> c(nm);
                for (int m = 0; m < nm; m++) {
                    c[m] = kact[m] ? -dv[m] : 0.0;
                    if (kact[m]) H[m][(size_t)k * (mk + 1) + i] = dv[m];
                }
                CK(axpby(w, one, w, c, vi));
            }
            CK(member_dots(w, w, dv));
            std::vector<double> sc(nm, 0.0);
            for (int m = 0; m < nm; m++) {
                if (!kact[m]) continue;
                double *hk = &H[m][(size_t)k * (mk + 1)];
                hk[k + 1] = std::sqrt(dv[m]);
                sc[m] = hk[k + 1] > 0.0 ? 1.0 / hk[k + 1] : 0.0;
                for (int i = 0; i < k; i++) {
                    const double t = cs[m][i] * hk[i] + sn[m][i] * hk[i + 1];
                    hk[i + 1] = -sn[m][i] * hk[i] + cs[m][i] * hk[i + 1];
                    hk[i] = t;
                }
                const double d = std::hypot(hk[k], hk[k + 1]);
                cs[m][k] = d == 0.0 ? 1.0 : hk[k] / d;
                sn[m][k] = d == 0.0 ? 0.0 : hk[k + 1] / d;
                hk[k] = d;
                hk[k + 1] = 0.0;
                gg[m][k + 1] = -sn[m][k] * gg[m][k];
                gg[m][k] = cs[m][k] * gg[m][k];
                kused[m] = k + 1;
                R[m].krylov_total++;
                if (std::fabs(gg[m][k + 1]) <= eta[m] * r[m] || d == 0.0 || k + 1 == mk) kact[m] = 0;
            }
            CK(axpby(V + (size_t)(k + 1) * len, sc, w, zero, w));
        }
        // step s = V y per member
        CK(cudaMemsetAsync(S, 0, sizeof(double) * len, s0));
        std::vector<std::vector<double>> yk(nm);
        for (int m = 0; m < nm; m++) {
            yk[m].assign(kused[m], 0.0);
            for (int i = kused[m] - 1; i >= 0; i--) {
                double s = gg[m][i];
                for (int jx = i + 1; jx < kused[m]; jx++) s -= H[m][(size_t)jx * (mk + 1) + i] * yk[m][jx];
                const double dii = H[m][(size_t)i * (mk + 1) + i];
                yk[m][i] = dii != 0.0 ? s / dii : 0.0;
            }
        }
        const int kmax = *std::max_element(kused.begin(), kused.end());
        for (int i = 0; i < kmax; i++) {
            std::vector<double> c(nm, 0.0);
            for (int m = 0; m < nm; m++) c[m] = i < kused[m] ? yk[m][i] : 0.0;
            CK(axpby(S, one, S, c, V + (size_t)i * len));
        }
        // zero-mass projection of every member's step
        k_member_mass<<<nm, 256, 0, s0>>>(S, vol, off_d, n, dots);
        std::vector<double> ms(nm);
        CK(cudaMemcpy(ms.data(), dots, sizeof(double) * nm, cudaMemcpyDeviceToHost));
        for (int m = 0; m < nm; m++) ms[m] /= wsum[m];
        CK(host_vec(ms, sc_a));
        k_member_sub_mass<<<grid, 256, 0, s0>>>(S, sc_a, vol, rm_d, n, len);
        CK(cudaGetLastError());
        // ---- line search per member, in lockstep
        std::vector<double> slope(nm), f0(nm), lam(nm, 0.0), lamp(nm, -1.0), fp(nm, 0.0), fn(nm, 0.0);
        std::vector<char> ls(nm, 0);
        for (int m = 0; m < nm; m++) {
            if (!act[m]) continue;
            const double rho = std::fabs(gg[m][kused[m]]);
            slope[m] = -(r[m] * r[m] - rho * rho);
            f0[m] = 0.5 * r[m] * r[m];
            lam[m] = 1.0;
            ls[m] = 1;
            R[m].krylov[std::min(R[m].newton_steps, M3D_NEWTON_MAX_HIST - 1)] = kused[m];
            R[m].etas[std::min(R[m].newton_steps, M3D_NEWTON_MAX_HIST - 1)] = eta[m];
            R[m].slopes[std::min(R[m].newton_steps, M3D_NEWTON_MAX_HIST - 1)] = slope[m];
        }
        // each member backtracks as the single solve does: a trial whose residual is not finite
        // gives no model and is cut to a tenth; no step below 1e-4 is tried, and a member whose
        // search fails keeps its iterate (lambda 0) and stops
        int trials = 0;
        std::vector<double> lam_eval(nm, -1.0);     // the step lengths of the last evaluated trial
        while (true) {
            bool anyls = false;
            for (int m = 0; m < nm; m++) {
                if (ls[m] && o.line_search && lam[m] < 1e-4) {
                    ls[m] = 0;
                    lam[m] = 0.0;
                    stopped[m] = 1;
                }
                anyls = anyls || ls[m];
            }
            if (!anyls) break;
            lam_eval = lam;
            CK(axpby(Yt, one, Y, lam, S));
            ST(phi(Yt, PYt));
            CK(axpby(tmp, one, Yt, mone, PYt));
            CK(member_dots(tmp, tmp, dv));
            trials++;
            for (int m = 0; m < nm; m++) {
                if (!ls[m]) continue;
                fn[m] = 0.5 * dv[m];
                if (R[m].ntrial < M3D_NEWTON_MAX_TRIALS) R[m].trial_lambdas[R[m].ntrial++] = lam[m];
                R[m].trials[std::min(R[m].newton_steps, M3D_NEWTON_MAX_HIST - 1)]++;
                if (!o.line_search) {
                    ls[m] = 0;
                    continue;
                }
                if (!std::isfinite(fn[m])) {
                    lamp[m] = -1.0;
                    lam[m] *= 0.1;
                    continue;
                }
                if (fn[m] <= f0[m] + 1e-4 * lam[m] * slope[m]) {
                    ls[m] = 0;
                    continue;
                }
                const double lt = lamp[m] < 0.0 ? quad_bt(f0[m], slope[m], lam[m], fn[m])
                                                : cubic_bt(f0[m], slope[m], lam[m], fn[m], lamp[m], fp[m]);
                lamp[m] = lam[m];
                fp[m] = fn[m];
                lam[m] = std::isfinite(lt) ? std::min(std::max(lt, 0.1 * lam[m]), 0.5 * lam[m]) : 0.1 * lam[m];
            }
            if (trials > 64) {              // not reached: lambda falls below 1e-4 within 14 trials
                for (int m = 0; m < nm; m++)
                    if (ls[m]) {
                        ls[m] = 0;
                        lam[m] = 0.0;
                        stopped[m] = 1;
                    }
                break;
            }
        }
        // accept: Y += lam S.  When the last trial evaluated every member at its accepted step
        // length, that trial is the new iterate and its year map is phi(Y) (the same kernels on
        // the same inputs, so the same bits); otherwise one more year map.
        if (lam_eval == lam) {
            CK(cudaMemcpyAsync(Y, Yt, sizeof(double) * len, cudaMemcpyDeviceToDevice, s0));
            CK(cudaMemcpyAsync(PY, PYt, sizeof(double) * len, cudaMemcpyDeviceToDevice, s0));
        } else {
            CK(axpby(Y, one, Y, lam, S));
            ST(phi(Y, PY));
        }
        CK(axpby(F, one, Y, mone, PY));
        CK(member_dots(F, F, dv));
        for (int m = 0; m < nm; m++) {
            if (!act[m]) continue;
            rprev[m] = r[m];
            etaprev[m] = eta[m];
            r[m] = std::sqrt(dv[m]);
            R[m].lambdas[std::min(R[m].newton_steps, M3D_NEWTON_MAX_HIST - 1)] = lam[m];
            if (stopped[m]) R[m].line_search_failed = 1;
            R[m].newton_steps++;
            R[m].residuals[std::min(R[m].newton_steps, M3D_NEWTON_MAX_HIST - 1)] = r[m];
        }
    }
#undef CK
#undef ST
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    bool all = true;
    for (int m = 0; m < nm; m++) {
        R[m].residual = r[m];
        R[m].converged = r[m] <= o.tol;
        R[m].year_maps = year_maps;
        R[m].tangent_maps = tangent_maps;
        R[m].seconds = secs;
        all = all && R[m].converged;
        if (reports) reports[m] = R[m];
    }
    return all ? M3D_OK : M3D_NOT_CONVERGED;
}
