// tmm_kernels.cuh -- device code of the TMM step (Metos3D, arXiv:1410.0204, Section 3):
//     y_{j+1} = A_imp(t_j) ( A_exp(t_j) y_j + q_j(y_j, u) ),
// fused into one pass per tile of water columns, and the year map of Section 4 as one
// persistent launch.  FP64 throughout.
//
// GB300 facts that shape this code: the FP64 pipe retires one warp-wide DFMA every 16
// clocks per SM (2 lanes per clock; measured 1.2 TFLOP/s for the GPU, 64x below FP32), and
// a warp instruction costs the same whether 1 or 32 lanes are active.  The year map is
// therefore bound by FP64 instruction issue, not by HBM.  Every FP64 instruction here is
// laid out so that all 32 lanes do useful work; scalars that need a division (the month
// weight, the internal step length) come precomputed; transcendentals are hoisted into
// per-init (insolation) and per-call (light attenuation, Martin profile) tables.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace m3d {

#ifndef M3D_THREADS
#define M3D_THREADS 512
#endif
constexpr int kThreads = M3D_THREADS; // threads per tile CTA (512: 16 warps, 4 per SM sub-partition)
// The resident year kernel splits its CTA: the last kQWarps warps evaluate the source term
// while the others wait for the neighbouring tiles and apply the explicit matrix.
constexpr int kQWarps = 4;
constexpr int kQThreads = kQWarps * 32;
constexpr int kSpThreads = kThreads - kQThreads;
static_assert(kSpThreads % 128 == 0, "the explicit group must span the four SM sub-partitions evenly");
constexpr int kModelNone = 0;
constexpr int kModelNdop = 2;
constexpr int kModelNdopTangent = 102;   // PO4-DOP with its tangent: state (N, DOP, dN, dDOP)
// The PO4-DOP model linearised about a trajectory recorded beforehand: state (dN, dDOP); the
// source term's Jacobian comes from the recorded df/dN of every euphotic cell and step.
constexpr int kModelNdopLinear = 103;
constexpr double kSigmaPar = 0.4;    // photosynthetically available fraction of I_SWR
constexpr int kEuphotic = 2;         // euphotic layers (Section 7: two)

// Scalars of the PO4-DOP model computed once per call from u (prologue kernel).
enum { kQAlpha = 0, kQSigma, kQLambda, kQKN, kQKI, kQOneMinusSigma, kQCount = 8 };

// One tile: a contiguous range of whole water columns, processed by one CTA.
struct Tile {
    int cell0, ncell;                // cells [cell0, cell0 + ncell)
    int sp0, sp1;                    // explicit-matrix warp slices [sp0, sp1)
    int bk0, bk1;                    // implicit-block warp slices [bk0, bk1)
    int eu0, eu1;                    // entries of eu_list: euphotic cells / shallow columns
    int ap0, ap1;                    // entries of ap_list: aphotic cells
    int sh0, sh1;                    // entries of sh_list: bottom cells of shallow columns (nsub = 1)
};

// Everything one step reads, as device pointers owned by the context.
struct StepParams {
    int n, nstep, nmonth, nsub, nulat, zmax;
    double ds;                             // internal model step, (1/nstep)/nsub
    const int *m0tab;                      // [nstep] first month of step j
    const double *wtab;                    // [nstep] interpolation weight of step j
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
    // slices of each tile dealt to its warps so that the four SM sub-partitions (warp w runs
    // on sub-partition w mod 4, each with its own FP64 unit) get equal FP64 work: the slices
    // of warp w of tile t are wlist[woff[t*(nwarps+1) + w] .. woff[t*(nwarps+1) + w + 1])
    const int *sp_wlist, *sp_woff, *bk_wlist, *bk_woff;
    // the same explicit slices dealt to the kSpThreads / 32 warps of the resident kernel's
    // explicit group: sp_wlist_g[sp_woff_g[t*(ng+1) + w] .. sp_woff_g[t*(ng+1) + w + 1])
    const int *sp_wlist_g, *sp_woff_g;
    const double *bk_b, *bk_d;             // [nmonth][...]: B_m and B_{m+1} - B_m
    long long bk_mstride;
    // The implicit part in Thomas form for the streaming kernels (use_tri != 0; at most two
    // tracers): factors [month][3][n] (-l_k, 1/d_k, -e_k/d_{k+1}), and per tile its (column,
    // tracer) chains packed as pack_chain(first tile-local cell, layers, tracer, 0), deepest first
    const double *tri;
    long long tri_mstride;
    const int *tchains, *tchain_off;       // [ntiles+1]
    int use_tri;
    // biogeochemistry
    const int *eu_list, *ap_list;          // tile-local cells, grouped per tile
    const int *sh_list;                    // tile-local bottom cells of shallow columns (nsub = 1)
    const int *cell_kl;                    // layer k | (column layers L << 8)
    const int *cell_ulat;                  // index of the cell's latitude in the insolation table
    const double *h;                       // [n] layer thickness
    const double *atten;                   // [n] sigma_PAR exp(-k_w d) (euphotic cells; per call)
    const double *mfrac;                   // [n] Martin deposition profile (aphotic cells; per call)
    const double *I0tab;                   // [nstep][nulat] daily-mean I_SWR at t_j
    const double *qpar;                    // [kQCount] model scalars (per call)
    // Linearisation of the PO4-DOP source term (one internal step): df/dN of every entry e of
    // eu_list at step j, [nstep][n_eu].  fn_out (null: not recorded) receives it while a year
    // map runs; the linearised year kernel reads fn_in.
    double *fn_out;
    const double *fn_in;
    int n_eu;
};

// Month weights (Section 3): month m is centred at t = (m + 1/2)/nmonth; t_j = j/nstep.
// s = nmonth t_j - 1/2 = num/den with num = 2 nmonth j - nstep, den = 2 nstep;
// m0 = floor(s) mod nmonth, w = s - floor(s) in [0, 1); the operator is M_m0 + w (M_m1 - M_m0).
// Evaluated once per step at set-up into m0tab/wtab.
__host__ __device__ inline void month_weights(int j, int nstep, int nmonth, int &m0, double &w)
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

// Dual numbers (value, directional derivative) for the tangent of the source term: the
// model functions below are templates over the scalar, so their tangent is the same code
// evaluated on dual numbers.
struct Dual {
    double v, d;
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.v * b.d + a.d * b.v}; }
__device__ __forceinline__ Dual operator*(double c, Dual a) { return {c * a.v, c * a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, double c) { return {a.v * c, a.d * c}; }
__device__ __forceinline__ Dual operator+(Dual a, double c) { return {a.v + c, a.d}; }
__device__ __forceinline__ Dual operator+(double c, Dual a) { return {c + a.v, a.d}; }
__device__ __forceinline__ Dual operator/(Dual a, double c) { return {a.v / c, a.d / c}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b)
{
    const double q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ Dual operator/(double c, Dual b)
{
    const double q = c / b.v;
    return {q, -(q * b.d) / b.v};
}
__device__ __forceinline__ Dual operator-(double c, Dual a) { return {c - a.v, -a.d}; }
__device__ __forceinline__ Dual operator-(Dual a, double c) { return {a.v - c, a.d}; }
__device__ __forceinline__ Dual &operator+=(Dual &a, Dual b) { a = a + b; return a; }

template <class T> __device__ __forceinline__ T zero_of();
template <> __device__ __forceinline__ double zero_of<double>() { return 0.0; }
template <> __device__ __forceinline__ Dual zero_of<Dual>() { return {0.0, 0.0}; }

// PO4-DOP euphotic cell over nsub internal steps (Section 2.2.1), light I fixed:
//   f = alpha N/(N+K_N) I/(I+K_I),  dN = -f + lambda DOP,  dDOP = sigma f - lambda DOP.
// Returns the increments and the production summed over the internal steps.  With one
// internal step the two Michaelis-Menten quotients share one division.
template <class T>
__device__ __forceinline__ void ndop_euphotic(T N, T D, double I, double alpha, double sigma, double lambda,
                                              double KN, double KI, double ds, int nsub, T &dN, T &dD, T &fsum)
{
    if (nsub == 1) {
        T f = (alpha * N * I) / ((N + KN) * (I + KI));
        T lD = lambda * D;
        dN = ds * (lD - f);
        dD = ds * (sigma * f - lD);
        fsum = f;
        return;
    }
    double aLF = alpha * (I / (I + KI));
    T N0 = N, D0 = D;
    fsum = zero_of<T>();
    for (int s = 0; s < nsub; s++) {
        T f = aLF * (N / (N + KN));
        T lD = lambda * D;
        N = N + ds * (lD - f);
        D = D + ds * (sigma * f - lD);
        fsum += f;
    }
    dN = N - N0;
    dD = D - D0;
}

// Aphotic PO4-DOP cell: DOP remineralises at lambda; the sinking flux deposits
// Esum * mfrac, Esum being the export summed over the internal steps.
template <class T>
__device__ __forceinline__ void ndop_aphotic(T D, T Esum, double mfrac, double lambda, double ds, int nsub, T &dN,
                                             T &dD)
{
    if (nsub == 1) {
        T lD = lambda * D;
        dN = ds * (lD + mfrac * Esum);
        dD = ds * (-lD);
        return;
    }
    T D0 = D, Dsum = zero_of<T>();
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
template <class T>
__device__ __forceinline__ void ndop_shallow_column(int L, const double *hcol, const T *N0, const T *D0,
                                                    const double *I, double alpha, double sigma, double lambda,
                                                    double KN, double KI, double ds, int nsub, T *dN, T *dD)
{
    T N[kEuphotic], D[kEuphotic];
    for (int k = 0; k < L; k++) { N[k] = N0[k]; D[k] = D0[k]; }
    for (int s = 0; s < nsub; s++) {
        T E = zero_of<T>(), f[kEuphotic];
        for (int k = 0; k < L; k++) {
            f[k] = alpha * (N[k] / (N[k] + KN)) * (I[k] / (I[k] + KI));
            E += (1.0 - sigma) * f[k] * hcol[k];
        }
        for (int k = 0; k < L; k++) {
            T qN = -f[k] + lambda * D[k];
            if (k == L - 1) qN += E / hcol[k];
            T qD = sigma * f[k] - lambda * D[k];
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

// Read access to a state vector: [tracer][cell] (the caller's layout) or [cell][tracer]
// (interleaved, used inside the resident year kernel so one gather serves all tracers).
template <int NTR, bool INTERLEAVED, bool COHERENT>
struct StateView {
    const double *y;
    int n;
    __device__ __forceinline__ double get(int cell, int t) const
    {
        const double *p = INTERLEAVED ? y + (size_t)cell * NTR + t : y + (size_t)t * n + cell;
        return load_state<COHERENT>(p);
    }
    __device__ __forceinline__ void gather(int cell, double *v) const
    {
        if (INTERLEAVED && NTR % 2 == 0) {
            const double *p = y + (size_t)cell * NTR;
#pragma unroll
            for (int t = 0; t < NTR; t += 2) {
                double2 q = COHERENT ? __ldcg(reinterpret_cast<const double2 *>(p + t))
                                     : __ldg(reinterpret_cast<const double2 *>(p + t));
                v[t] = q.x;
                v[t + 1] = q.y;
            }
        } else {
#pragma unroll
            for (int t = 0; t < NTR; t++) v[t] = get(cell, t);
        }
    }
};

// Barriers: 0, the whole CTA; 1, its first kThreads - 32 threads; 2, its last kQThreads
// threads (the source-term group); 3, its first kSpThreads threads (the explicit group).
__device__ __forceinline__ void barrier_sub(int id)
{
    if (id == 0) __syncthreads();
    else if (id == 1) asm volatile("bar.sync 1, %0;" :: "n"(kThreads - 32) : "memory");
    else if (id == 2) asm volatile("bar.sync 2, %0;" :: "n"(kQThreads) : "memory");
    else asm volatile("bar.sync 3, %0;" :: "n"(kSpThreads) : "memory");
}

// Access to the model state of one cell as a scalar (N or DOP) or, for the tangent, as a
// dual number (N, dN) or (DOP, dDOP) from components (0, 2) and (1, 3).
template <class T> struct ModelState;
template <> struct ModelState<double> {
    template <class SV> __device__ __forceinline__ static double get(const SV &Y, int cell, int which)
    {
        return Y.get(cell, which);
    }
    __device__ __forceinline__ static void put(double *dq, int zmax, int i, int which, double v) { dq[which * zmax + i] = v; }
    __device__ __forceinline__ static void add(double *dq, int zmax, int i, int which, double v) { dq[which * zmax + i] += v; }
    __device__ __forceinline__ static void put_e(double *ek, int zmax, int i, double v) { ek[i] = v; }
    __device__ __forceinline__ static double get_e(const double *ek, int zmax, int i) { return ek[i]; }
};
template <> struct ModelState<Dual> {
    template <class SV> __device__ __forceinline__ static Dual get(const SV &Y, int cell, int which)
    {
        return {Y.get(cell, which), Y.get(cell, which + 2)};
    }
    __device__ __forceinline__ static void put(double *dq, int zmax, int i, int which, Dual v)
    {
        dq[which * zmax + i] = v.v;
        dq[(which + 2) * zmax + i] = v.d;
    }
    __device__ __forceinline__ static void add(double *dq, int zmax, int i, int which, Dual v)
    {
        dq[which * zmax + i] += v.v;
        dq[(which + 2) * zmax + i] += v.d;
    }
    __device__ __forceinline__ static void put_e(double *ek, int zmax, int i, Dual v)
    {
        ek[i] = v.v;
        ek[zmax + i] = v.d;
    }
    __device__ __forceinline__ static Dual get_e(const double *ek, int zmax, int i) { return {ek[i], ek[zmax + i]}; }
};

// Whether the source term of scalar type T records its Jacobian for a linearised sweep (the
// plain model does; its tangent on dual numbers does not).
template <class T> struct ModelTraits_record { static constexpr bool ok = false; };
template <> struct ModelTraits_record<double> {
    static constexpr bool ok = true;
    __device__ __forceinline__ static double value(double v) { return v; }
};

// The source-minus-sink increment of the PO4-DOP model (Section 2.2.1) for every cell of a
// tile, computed from y_j and written to dq[t * zmax + i].  Reads only the tile's own cells.
// Run by threads [tid0, tid0 + nthr) of the CTA, which synchronise on barrier `bar`:
// euphotic cells first, then aphotic cells (which need their column's export) and the
// export kept in the bottom layer of shallow columns.  With several internal steps a
// shallow column runs whole on one thread, since its cells then couple at every step.
// T = double: the model; T = Dual: the model and its tangent (ek then holds 2 * zmax).
template <class T, class SV>
__device__ __forceinline__ void ndop_source_tile(const StepParams &P, const Tile &T_, int j, const SV &Y,
                                                 double *dq, double *ek, int nthr, int bar, int tid0 = 0)
{
    typedef ModelState<T> MS;
    const int tid = (int)threadIdx.x - tid0;
    const int zmax = P.zmax;
    const double alpha = __ldg(P.qpar + kQAlpha), sigma = __ldg(P.qpar + kQSigma);
    const double lambda = __ldg(P.qpar + kQLambda), KN = __ldg(P.qpar + kQKN);
    const double KI = __ldg(P.qpar + kQKI), oms = __ldg(P.qpar + kQOneMinusSigma);
    const int nsub = P.nsub;
    const double ds = P.ds;
    const double *I0row = P.I0tab + (size_t)j * P.nulat;
    for (int e = T_.eu0 + tid; e < T_.eu1; e += nthr) {
        const int i = __ldg(P.eu_list + e);
        const int cell = T_.cell0 + i;
        const int L = __ldg(P.cell_kl + cell) >> 8;
        const double I0 = __ldg(I0row + __ldg(P.cell_ulat + cell));
        if (L <= kEuphotic && nsub > 1) {
            T N0[kEuphotic], D0[kEuphotic], dN[kEuphotic], dD[kEuphotic];
            double I[kEuphotic];
            for (int kk = 0; kk < L; kk++) {
                N0[kk] = MS::get(Y, cell + kk, 0);
                D0[kk] = MS::get(Y, cell + kk, 1);
                I[kk] = I0 * __ldg(P.atten + cell + kk);
            }
            ndop_shallow_column<T>(L, P.h + cell, N0, D0, I, alpha, sigma, lambda, KN, KI, ds, nsub, dN, dD);
            for (int kk = 0; kk < L; kk++) {
                MS::put(dq, zmax, i + kk, 0, dN[kk]);
                MS::put(dq, zmax, i + kk, 1, dD[kk]);
            }
        } else {
            T dN, dD, fsum;
            const double I = I0 * __ldg(P.atten + cell);
            ndop_euphotic<T>(MS::get(Y, cell, 0), MS::get(Y, cell, 1), I, alpha, sigma,
                             lambda, KN, KI, ds, nsub, dN, dD, fsum);
            if constexpr (ModelTraits_record<T>::ok) {
                if (P.fn_out && nsub == 1) {
                    // df/dN = alpha I K_N / ((N + K_N)^2 (I + K_I)), the Jacobian a linearised sweep needs
                    const double N = ModelTraits_record<T>::value(MS::get(Y, cell, 0));
                    const double d = N + KN;
                    P.fn_out[(size_t)j * P.n_eu + e] = (alpha * I * KN) / (d * d * (I + KI));
                }
            }
            MS::put(dq, zmax, i, 0, dN);
            MS::put(dq, zmax, i, 1, dD);
            MS::put_e(ek, zmax, i, oms * fsum * __ldg(P.h + cell));
        }
    }
    barrier_sub(bar);
    for (int a = T_.ap0 + tid; a < T_.ap1; a += nthr) {
        const int i = __ldg(P.ap_list + a);
        const int cell = T_.cell0 + i;
        const int k = __ldg(P.cell_kl + cell) & 0xff;
        const T Esum = MS::get_e(ek, zmax, i - k) + MS::get_e(ek, zmax, i - k + 1);
        T dN, dD;
        ndop_aphotic<T>(MS::get(Y, cell, 1), Esum, __ldg(P.mfrac + cell), lambda, ds, nsub, dN, dD);
        MS::put(dq, zmax, i, 0, dN);
        MS::put(dq, zmax, i, 1, dD);
    }
    // shallow columns (one internal step): the export stays in the bottom layer
    for (int b = T_.sh0 + tid; b < T_.sh1; b += nthr) {
        const int i = __ldg(P.sh_list + b);
        const int cell = T_.cell0 + i;
        const int k = __ldg(P.cell_kl + cell) & 0xff;
        const T Esum = (k == 0) ? MS::get_e(ek, zmax, i) : MS::get_e(ek, zmax, i - 1) + MS::get_e(ek, zmax, i);
        MS::add(dq, zmax, i, 0, ds * (Esum / __ldg(P.h + cell)));
    }
}

// The PO4-DOP increment linearised about a recorded trajectory (one internal step): for the
// perturbation (dN, dDOP) of y_j, with f_N = df/dN recorded at step j,
//   euphotic: df = f_N dN,  d(dq_N) = ds (lambda dDOP - df),  d(dq_DOP) = ds (sigma df - lambda dDOP),
//   export:   dE = (1 - sigma) sum over the column's euphotic cells of df h,
//   aphotic:  d(dq_N) = ds (lambda dDOP + mfrac dE),  d(dq_DOP) = -ds lambda dDOP,
//   shallow column: its bottom layer also gets ds dE / h.
// The same structure and threads as ndop_source_tile.
template <class SV>
__device__ __forceinline__ void ndop_source_tile_linear(const StepParams &P, const Tile &T_, int j, const SV &Y,
                                                        double *dq, double *ek, int nthr, int bar, int tid0 = 0)
{
    const int tid = (int)threadIdx.x - tid0;
    const int zmax = P.zmax;
    const double sigma = __ldg(P.qpar + kQSigma), lambda = __ldg(P.qpar + kQLambda);
    const double oms = __ldg(P.qpar + kQOneMinusSigma);
    const double ds = P.ds;
    const double *fn = P.fn_in + (size_t)j * P.n_eu;
    for (int e = T_.eu0 + tid; e < T_.eu1; e += nthr) {
        const int i = __ldg(P.eu_list + e);
        const int cell = T_.cell0 + i;
        const double dN = Y.get(cell, 0), dD = Y.get(cell, 1);
        const double df = __ldg(fn + e) * dN;
        const double lD = lambda * dD;
        dq[i] = ds * (lD - df);
        dq[zmax + i] = ds * (sigma * df - lD);
        ek[i] = oms * df * __ldg(P.h + cell);
    }
    barrier_sub(bar);
    for (int a = T_.ap0 + tid; a < T_.ap1; a += nthr) {
        const int i = __ldg(P.ap_list + a);
        const int cell = T_.cell0 + i;
        const int k = __ldg(P.cell_kl + cell) & 0xff;
        const double Esum = ek[i - k] + ek[i - k + 1];
        const double lD = lambda * Y.get(cell, 1);
        dq[i] = ds * (lD + __ldg(P.mfrac + cell) * Esum);
        dq[zmax + i] = ds * (-lD);
    }
    for (int b = T_.sh0 + tid; b < T_.sh1; b += nthr) {
        const int i = __ldg(P.sh_list + b);
        const int cell = T_.cell0 + i;
        const int k = __ldg(P.cell_kl + cell) & 0xff;
        const double Esum = (k == 0) ? ek[i] : ek[i - 1] + ek[i];
        dq[i] += ds * (Esum / __ldg(P.h + cell));
    }
}

// Whether a model has a source term, and its scalar type.
template <int MODEL> struct ModelTraits { static constexpr bool has_q = false; typedef double scalar; };
template <> struct ModelTraits<kModelNdop> { static constexpr bool has_q = true; typedef double scalar; };
template <> struct ModelTraits<kModelNdopTangent> { static constexpr bool has_q = true; typedef Dual scalar; };
template <> struct ModelTraits<kModelNdopLinear> { static constexpr bool has_q = true; typedef double scalar; };

// One TMM step on one tile.  smem: (NTR + 2) * zmax doubles.
// Order: q increment of the tile's own cells into z (no neighbour data needed), then
// z += A_exp(t_j) y_j, then y_{j+1} = A_imp(t_j) z.
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
    double *z = smem;                 // [NTR][zmax] dq, then A_exp y + dq, tile-local cells
    double *ek = smem + NTR * zmax;   // [2 zmax] export contributions of euphotic cells (and tangent)

    const int m0 = __ldg(P.m0tab + j);
    const double w = __ldg(P.wtab + j);

    // ---- source-minus-sink increment on y_j (Section 2.2.1)
    if (ModelTraits<MODEL>::has_q) {
        StateView<NTR, false, COHERENT> Y{y, n};
        ndop_source_tile<typename ModelTraits<MODEL>::scalar>(P, T, j, Y, z, ek, blockDim.x, 0);
        __syncthreads();
    }

    // ---- explicit part: z += (A_m0 + w (A_m1 - A_m0)) y, all tracers per matrix read
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
                for (int t = 0; t < NTR; t++)
                    z[t * zmax + row] = ModelTraits<MODEL>::has_q ? acc[t] + z[t * zmax + row] : acc[t];
            }
        }
    }
    __syncthreads();

    // ---- implicit part in Thomas form: y_{j+1} = (1 - w) M_m0^{-1} z + w M_m1^{-1} z, one
    // thread per (column, tracer) solving both months in turn with the factors read from
    // global memory (the tile's shared memory holds z and, in the export scratch no longer
    // needed, the forward sweep's intermediates).  Month m1 first: its weighted solution
    // c1 u1 is stored, then month m0 adds c0 u0 with one fused multiply-add, as the resident
    // kernel's blend does, so both give the same bits.
    if constexpr (NTR <= 2) {
        if (P.use_tri) {
            const int m1 = (m0 + 1) % P.nmonth;
            const int c0 = __ldg(P.tchain_off + tile), c1 = __ldg(P.tchain_off + tile + 1);
            for (int c = c0 + (int)threadIdx.x; c < c1; c += blockDim.x) {
                const int pc = __ldg(P.tchains + c);
                const int cb = pc & 0xffff, L = (pc >> 16) & 0x7f, t = (pc >> 23) & 0xf;
                const int cell = T.cell0 + cb;
                const double *zc = z + t * zmax + cb;
                double *g = ek + t * zmax + cb;
                double *out = yn + (size_t)t * n + cell;
                for (int h = 1; h >= 0; h--) {
                    const double *F = P.tri + (long long)(h ? m1 : m0) * P.tri_mstride + cell;
                    const double *nl = F, *rd = F + n, *ne = F + 2 * (size_t)n;
                    const double wt = h ? w : 1.0 - w;
                    double acc = 0.0;
                    for (int k = 0; k < L; k++) {            // g_k = z_k - l_k g_{k-1}
                        acc = fma(__ldg(nl + k), acc, zc[k]);
                        g[k] = acc;
                    }
                    double u = 0.0;
                    for (int k = L - 1; k >= 0; k--) {       // u_k = g_k - (e_k/d_{k+1}) u_{k+1}
                        u = fma(__ldg(ne + k), u, g[k]);
                        const double cw = wt * __ldg(rd + k);
                        out[k] = h ? cw * u : fma(cw, u, out[k]);
                    }
                }
            }
            return;
        }
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

// ------------------------------------------------------------------------------------------
// Persistent year map: one cooperative launch, one CTA per tile, all tiles co-resident.
// Before step s a tile waits until every tile it reads from, or that reads from it, has
// finished step s-1 (per-tile counters, release/acquire at GPU scope).  That makes y_s
// complete where this tile reads it, and makes the buffer it overwrites (y_{s-1}) no longer
// read by anyone.  Every wait is bounded: after timeout_ns the tile records the failure in
// status[] and returns, and the others stop at their next wait.

struct SyncParams {
    int *flags;                 // [ntiles] steps completed (0 at launch)
    const int *dep_off;         // [ntiles+1]
    const int *dep_idx;         // neighbour tiles
    int *status;                // [4]: 0 ok / 1 timeout; tile; step; 1 if an aborting tile's own copy did not land
    unsigned long long timeout_ns;
    int withhold_tile;          // test hook: this tile never publishes its counter (-1: none)
    // Non-null: a device flag set by an earlier kernel on the same stream; when it is nonzero
    // at launch the year kernels return at once (every tile reads the same value).  A Krylov
    // solve that enqueues its iterations ahead of its convergence test uses it to skip the
    // iterations enqueued after convergence.
    const int *skip;
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int load_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void store_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Release-ordered add (gpu scope): the calling thread's earlier writes, and those ordered before
// them by a barrier it took part in, are visible to whoever acquires the new value.
__device__ __forceinline__ void add_release(int *p, int v)
{
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Warp 0 waits for the neighbours of `tile` to reach `target`; returns false on abort.
__device__ __forceinline__ bool wait_neighbours(const SyncParams &S, int tile, int target, int step)
{
    const int lane = threadIdx.x & 31;
    bool ok = true;
    const int d0 = __ldg(S.dep_off + tile), d1 = __ldg(S.dep_off + tile + 1);
    for (int d = d0 + lane; d < d1 && ok; d += 32) {
        const int nb = __ldg(S.dep_idx + d);
        if (load_acquire(S.flags + nb) >= target) continue;
        const unsigned long long t0 = global_ns();
        while (true) {
            if (load_acquire(S.flags + nb) >= target) break;
            if (*(volatile int *)S.status != 0) { ok = false; break; }
            if (global_ns() - t0 > S.timeout_ns) {
                if (atomicCAS(S.status, 0, 1) == 0) {
                    S.status[1] = tile;
                    S.status[2] = step;
                }
                ok = false;
                break;
            }
            __nanosleep(64);
        }
    }
    return __all_sync(0xffffffffu, ok);
}

template <int NTR, int MODEL>
__device__ __forceinline__ void year_persistent(const StepParams &P, const SyncParams &S,
                                                double *buf0, double *buf1, int j0, int nsteps,
                                                double *smem)
{
    __shared__ int abort_flag;
    const int tile = blockIdx.x;
    for (int s = 0; s < nsteps; s++) {
        const int j = (j0 + s) % P.nstep;
        const double *y = (s & 1) ? buf1 : buf0;
        double *yn = (s & 1) ? buf0 : buf1;
        if (s > 0) {
            if (threadIdx.x < 32) {
                bool ok = wait_neighbours(S, tile, s, s);
                if (threadIdx.x == 0) abort_flag = ok ? 0 : 1;
            }
            __syncthreads();
            if (abort_flag) return;
        }
        step_tile<NTR, MODEL, true>(P, tile, j, y, yn, smem);
        // the CTA barrier orders every thread's stores of y_{j+1} before thread 0's release
        __syncthreads();
        if (threadIdx.x == 0 && tile != S.withhold_tile) store_release(S.flags + tile, s + 1);
    }
}

}  // namespace m3d
