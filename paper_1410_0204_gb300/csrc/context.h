// context.h -- the library context shared by the translation units of libmetos3d (internal).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "metos3d.h"
#include "tmm_kernels.cuh"
#include "tmm_resident.cuh"

using m3d::StepParams;
using m3d::Tile;

typedef void (*step_kernel_t)(StepParams, int, const double *, double *);
typedef void (*year_kernel_t)(StepParams, m3d::SyncParams, double *, double *, int, int);
typedef void (*resident_kernel_t)(StepParams, m3d::ResidentParams, m3d::SyncParams, double *, long long, int, int,
                                  int);
typedef void (*layout_kernel_t)(int, const double *, double *);

struct ResidentKernels {
    resident_kernel_t year, year_tri;
    layout_kernel_t to_interleaved, from_interleaved;
};

// One way of running the year: the forward model, or the model with its tangent (twice the
// tracers).  Kernels, their shared memory, and which plans fit on the GPU.
struct YearVariant {
    int ntr = 0;
    int model = 0;                      // m3d::kModel*
    step_kernel_t step = nullptr;
    year_kernel_t year = nullptr;
    ResidentKernels rk{};
    size_t smem = 0, resident_smem = 0, resident_tri_smem = 0;
    int persistent_ok = 0, resident_ok = 0, tri_resident_ok = 0;
};

struct m3d_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int n = 0, ncol = 0, ntr = 0, nparam = 0, nsub = 1, nstep = 0, nmonth = 0, model = 0;
    int ntiles = 0, zmax = 0, nulat = 0;
    size_t smem_bytes = 0;
    std::vector<void *> allocs;
    StepParams P{};
    m3d::SyncParams S{};
    step_kernel_t step_kernel = nullptr;
    year_kernel_t year_kernel = nullptr;
    int plan = 0;                       // M3D_PLAN_*
    int persistent_ok = 0;              // all tiles fit on the GPU at once (streaming plan)
    int resident_ok = 0;                // ... with their month of matrices in shared memory
    int tri_ok = 0;                     // every implicit block is the inverse of a tridiagonal matrix
    int tri_resident_ok = 0;            // ... and the tridiagonal resident kernel fits
    int implicit_form = 0;              // M3D_IMPLICIT_DENSE or M3D_IMPLICIT_TRIDIAGONAL (resident plan)
    m3d::ResidentParams R{};
    ResidentKernels rk{};
    size_t resident_smem = 0, resident_tri_smem = 0;
    // adjoint: transposed operators (same layouts), its tables and kernels' shared memory
    int adj_ok = 0, adj_tri_ok = 0, adj_dense_ok = 0;
    int adj_stream_ok = 0;              // the streaming reverse sweep fits (operators read from HBM)
    int adj_force_stream = 0;           // M3D_OPT_ADJOINT_PLAN = M3D_PLAN_PERSISTENT
    double *sp_b = nullptr;             // per-step explicit operators [nstep][slot-lanes] (or null)
    int tri_stream_ok = 0;              // the streaming kernels can apply the Thomas form (<= 2 tracers)
    size_t sp_b_bytes = 0;
    double *spT_b = nullptr;            // the transposed per-step operators of the reverse sweep (or null)
    size_t spT_b_bytes = 0;
    size_t adj_smem_stream = 0;
    StepParams PT{};
    m3d::ResidentParams RTadj{};
    m3d::AdjointParams A{};
    size_t adj_smem_dense = 0, adj_smem_tri = 0;
    double *mfrac_b = nullptr;
    // PO4-DOP linearised about a recorded trajectory (one internal step, resident plan): the
    // linearised year kernels, whether they fit, which form metos3d_year_tangent uses, and the
    // recorded df/dN of metos3d_year_tangent's own forward pass ([nstep][n_eu], made on demand)
    ResidentKernels rk_lin{};
    int lin_ok = 0, lin_tri_ok = 0;
    int tangent_form = 0;               // M3D_TANGENT_DUAL or M3D_TANGENT_LINEARISED
    double *fn_buf = nullptr;
    YearVariant tan;                    // the model with its tangent (PO4-DOP only)
    m3d::ResidentParams R_tan{};        // resident layout of the tangent (its own Thomas chains)
    int tan_ok = 0;
    int *status_host = nullptr;         // pinned copy of S.status
    double *qpar = nullptr;
    double *u_dev = nullptr;
    double *ybuf[2] = {nullptr, nullptr};   // ybuf[1] = ybuf[0] + ybuf_cap (one allocation)
    long long ybuf_cap = 0;
    double *atten = nullptr, *mfrac = nullptr;
    double *vol = nullptr, *h = nullptr, *zc = nullptr;
    int *cell_kl = nullptr;
    double *red_part = nullptr, *red_out = nullptr, *red_host = nullptr;
    cudaGraphExec_t year_graph = nullptr;
    int year_result_buf = 0;
    long long last_launches = 0;
    cudaEvent_t kev[2] = {nullptr, nullptr};   // around the last year-kernel launch (M3D_OPT_KERNEL_TIMING)
    int time_kernel = 0, kev_recorded = 0;
    std::string err;
    // models only ensembles run (N, PO4-DOP-PHY, NPZD-DOP): a one-member ensemble does the steps
    m3d_ensemble *ens = nullptr;
    std::vector<double> ens_u;          // the parameters last given to it
    int ens_u_valid = 0;
    // ... and its tangent: a one-member tangent ensemble (state and perturbation), the
    // parameters last given to it, and a staging pair of [2 ntracer][n] arrays
    m3d_ensemble *ens_tan = nullptr;
    std::vector<double> ens_tan_u;
    int ens_tan_u_valid = 0;
    double *tan_buf = nullptr;
};

// Record a failure on c (or for metos3d_init when c is null) and return s.
m3d_status fail(m3d_ctx *c, m3d_status s, const char *fmt, ...);

#define CUDA_OR_FAIL(ctx, call)                                                              \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((ctx), M3D_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Internal entry points shared between translation units.
// The year map from the device state y0 to y1 with the parameters already in c->u_dev.
m3d_status m3d_year_device(m3d_ctx *c, const double *y0, double *y1);
// Copy nparam parameters into c->u_dev (kind: cudaMemcpyDeviceToDevice or HostToDevice).
m3d_status m3d_set_params(m3d_ctx *c, const double *u, cudaMemcpyKind kind);
// phi(y0) and phi'(y0) v with the parameters already in c->u_dev.
m3d_status m3d_year_tangent_device(m3d_ctx *c, const double *y0, const double *v, double *phi, double *jv);
// The year map recording df/dN of every euphotic cell and step into fn ([nstep][n_eu]); the
// linearised year map phi'(y) v about the trajectory recorded in fn (c->lin_ok contexts).
m3d_status m3d_year_record_device(m3d_ctx *c, const double *y0, double *y1, double *fn);
m3d_status m3d_year_linear_device(m3d_ctx *c, const double *fn, const double *v, double *jv);
// One TMM step j in the caller's layout (the step kernel; parameters already in c->u_dev and
// the per-call tables made).
m3d_status m3d_step_device(m3d_ctx *c, int j, const double *y, double *yn);
// Builds the reverse sweep's per-step transposed explicit operators (A_j^T for every step j,
// in the transposed slices' layout) the first time a resident reverse sweep runs, where the
// context keeps forward per-step operators and the device has room for a second array.
// Synchronous.  Leaves them absent (the sweep then interpolates in the kernel) otherwise.
m3d_status m3d_adjoint_step_operators(m3d_ctx *c);
// An ensemble-backed context (N, PO4-DOP-PHY, NPZD-DOP): hand the parameters in c->u_dev to its
// one-member ensemble (synchronous; nothing to do when they did not change).
m3d_status m3d_ens_sync_params(m3d_ctx *c);
// The per-call model tables (attenuation, Martin profile, model scalars) from c->u_dev.
m3d_status m3d_prologue(m3d_ctx *c);
// Device allocation owned by the context (freed by metos3d_free).
cudaError_t m3d_alloc(m3d_ctx *c, void **p, size_t bytes);
// The adjoint year map as one forward sweep and any number of reverse sweeps at the same
// (y0, u).  The forward sweep keeps a checkpoint every K steps (K >= nstep: the whole
// trajectory); each reverse sweep recomputes the K-step segments it needs that are not held
// (none when K >= nstep) and returns ybar0 = phi_y^T ybar1 and ubar = phi_u^T ybar1.  So
// repeated products phi_y^T v at one state, as a Krylov solve makes, cost one reverse sweep
// each after the first forward sweep.  PO4-DOP only (the caller checks c->adj_ok or
// c->adj_stream_ok through begin()).
struct AdjointSweep {
    m3d_ctx *c = nullptr;
    int K = 0, nseg = 0, held = -1;     // held: the segment whose states traj holds
    bool stream = false, tri = false;
    long long len = 0;
    double *traj = nullptr, *chk = nullptr, *zb = nullptr, *yb = nullptr;
    long long launches = 0;             // kernel launches so far
    long long forward_steps = 0;        // TMM steps run forward (first sweep and recomputations)
    int reverse_sweeps = 0;
    m3d_status begin(m3d_ctx *ctx, int ckpt_every);   // checks, then allocates the buffers
    m3d_status forward(const double *y0, const double *u);
    m3d_status reverse(const double *ybar1, double *ybar0, double *ubar_host);
    void release();
};
// Checks of a grid and its matrices (sizes, CSR order and range, block sizes, finiteness).
m3d_status m3d_validate_inputs(const m3d_grid *g, const m3d_matrices *mt, std::string &why);
// Thomas factors of M when the row-major L x L block B is M's inverse and M is tridiagonal.
bool tridiagonal_factors(const double *B, int L, double *nl, double *rd, double *ne);
// The resident kernels' form of one month of factors [3][n]: -e_k/d_k becomes -e_k/d_{k+1}.
void thomas_backsubstitution_form(double *tri_month, int n, const int *col_start, int ncol);
