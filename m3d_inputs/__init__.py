"""Seeded synthetic inputs for the Transport Matrix Method year map.

The paper's workloads (Section 7) use MITgcm-derived monthly transport matrices on a
2.8125 degree grid with 15 layers (52749 wet cells per tracer) and a 1 degree grid.
Those matrices are not available, so this module builds seeded stand-ins with the same
shape and structure:

* a lon-lat grid with a smooth seeded land mask and bathymetry (columns of 1..nz layers);
* twelve monthly explicit matrices ``A_exp,m = I + dt * L_m`` in CSR form with one shared
  sparsity pattern, where ``L_m`` is upwind advection by a divergence-free layer flow
  (from a streamfunction on cell corners) plus symmetric diffusive exchange with the
  4 face neighbours, the 4 diagonal neighbours, optionally the 4 distance-2 neighbours,
  and the 2 vertical neighbours -- all in flux form, so that ``V^T A = V^T`` and
  ``A 1 = 1``;
* twelve monthly implicit matrices ``A_imp,m = blockdiag_c (I - dt K_{m,c})^{-1}`` with
  ``K`` a tridiagonal vertical diffusion in flux form (so ``V^T A_imp = V^T`` and
  ``A_imp 1 = 1``), stored as one dense row-major ``L_c x L_c`` block per water column;
* the per-column latitude used for the insolation forcing, and the default parameters
  and initial state of the N-DOP model (Section 2.2.1).

Nothing in this module performs a step of the method: there is no time stepping, no
interpolation in time and no biogeochemical source term here.  It only builds inputs,
which the CPU oracle and the CUDA library both consume.

Random streams: every draw comes from ``numpy.random.Generator(PCG64)`` seeded with
``[seed, stream_id]`` for a named stream (mask, bathymetry, psi, kappa_h, kappa_v,
ensemble, observations), so that changing one ingredient does not shift the others.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Problem", "GridSpec", "SPECS", "make_problem", "spec", "default_params_ndop",
    "initial_state", "rng", "NDOP_PARAM_NAMES", "MODEL_NONE", "MODEL_NDOP",
    "MODEL_N", "MODEL_PHY", "MODEL_NPZD", "MODELS", "default_params", "model_initial_values",
    "Member", "make_ensemble", "ENSEMBLE_MIX",
]

EARTH_RADIUS = 6.371e6          # m
SECONDS_PER_YEAR = 360 * 86400  # the interface assumes a 360-day year (Section 5.1)

# Model identifiers shared by both sides of the boundary.
MODEL_NONE = 0   # q = 0: pure transport
MODEL_N = 1      # PO4 alone, all production exported (1 tracer)
MODEL_NDOP = 2   # the PO4-DOP model of Section 2.2.1 (2 tracers)
MODEL_PHY = 3    # the PO4-DOP-PHY model of Section 2.2.2 (3 tracers)
MODEL_NPZD = 5   # NPZD-DOP: PO4-DOP-PHY extended by zooplankton and sinking detritus (5 tracers)

# Parameter order of the N-DOP model: k_w [1/m], alpha [1/d], sigma [-], lambda [1/yr],
# K_N [mmol P/m^3], K_I [W/m^2], b [-].
NDOP_PARAM_NAMES = ("k_w", "alpha", "sigma", "lambda", "K_N", "K_I", "b")


@dataclasses.dataclass(frozen=True)
class ModelSpec:
    """Tracer names, parameter names (in order), default parameters, fractions among them."""
    model: int
    tracers: tuple
    params: tuple
    defaults: tuple
    fractions: tuple          # parameters that are fractions in [0, 1]
    initial: tuple            # spatially constant initial value of each tracer


MODELS = {
    MODEL_N: ModelSpec(MODEL_N, ("PO4",), ("k_w", "alpha", "K_N", "K_I", "b"),
                       (0.02, 0.5, 0.5, 30.0, 0.858), (), (2.17,)),
    MODEL_NDOP: ModelSpec(MODEL_NDOP, ("PO4", "DOP"), NDOP_PARAM_NAMES,
                          (0.02, 0.5, 0.67, 0.5, 0.5, 30.0, 0.858), ("sigma",), (2.17, 1.0e-4)),
    # order of the paper's parameter table (Section 2.2.2); rates per day
    MODEL_PHY: ModelSpec(MODEL_PHY, ("PO4", "DOP", "PHY"),
                         ("mu_1", "k_w", "K_1", "K_I", "lambda_2", "sigma_2", "lambda_3", "kappa_3",
                          "lambda_3p", "sigma_3", "b"),
                         (2.0, 0.02, 0.5, 30.0, 0.01, 0.67, 0.03, 1.0, 0.01, 0.75, 0.858),
                         ("sigma_2", "sigma_3"), (2.17, 1.0e-4, 0.01)),
    # rates per day, sinking speed in m/day
    MODEL_NPZD: ModelSpec(MODEL_NPZD, ("PO4", "PHY", "ZOO", "DET", "DOP"),
                          ("k_w", "mu_P", "K_N", "K_I", "mu_Z", "K_P", "epsilon", "lambda_P",
                           "kappa_Z", "lambda_Z", "lambda_D", "lambda_DOP", "w_D"),
                          (0.02, 1.0, 0.5, 30.0, 1.0, 0.1, 0.75, 0.05, 1.0, 0.03, 0.05, 0.01, 2.0),
                          ("epsilon",), (2.17, 0.01, 0.01, 0.01, 1.0e-4)),
}


def default_params(model: int) -> np.ndarray:
    """Default parameters u of a model, in its parameter order."""
    return np.array(MODELS[model].defaults, dtype=np.float64)


def model_initial_values(model: int) -> tuple:
    return MODELS[model].initial


@dataclasses.dataclass(frozen=True)
class Member:
    """One ensemble member: a model and its parameter vector."""
    model: int
    u: np.ndarray

    @property
    def ntracer(self) -> int:
        return len(MODELS[self.model].tracers)


# The batched ensemble: 16 runs of the N model, 32 of N-DOP, 16 of NPZD-DOP.
ENSEMBLE_MIX = ((MODEL_N, 16), (MODEL_NDOP, 32), (MODEL_NPZD, 16))


def make_ensemble(mix=ENSEMBLE_MIX, seed: int = 1410, spread: float = 0.5) -> list:
    """Members with parameters drawn uniformly within +-spread of each model's defaults.

    Draws come from the "ensemble" stream, members in the order of ``mix``; a parameter
    that is a fraction is capped at 1.
    """
    r = rng(seed, "ensemble")
    out = []
    for model, count in mix:
        sp = MODELS[model]
        base = np.array(sp.defaults, dtype=np.float64)
        frac = np.array([p in sp.fractions for p in sp.params])
        for _ in range(count):
            u = base * (1.0 + spread * (2.0 * r.random(base.size) - 1.0))
            u[frac] = np.minimum(u[frac], 1.0)
            out.append(Member(model, u))
    return out

_STREAMS = {"mask": 1, "bathymetry": 2, "psi": 3, "kappa_h": 4, "kappa_v": 5,
            "ensemble": 6, "observations": 7, "state": 8}


def rng(seed: int, stream: str) -> np.random.Generator:
    """The named, independent random stream ``stream`` of master seed ``seed``."""
    return np.random.Generator(np.random.PCG64([int(seed), _STREAMS[stream]]))


def default_params_ndop() -> np.ndarray:
    """Default N-DOP parameters u, in ``NDOP_PARAM_NAMES`` order."""
    return np.array([0.02, 0.5, 0.67, 0.5, 0.5, 30.0, 0.858], dtype=np.float64)


@dataclasses.dataclass(frozen=True)
class GridSpec:
    """Shape of one synthetic workload."""
    name: str
    nx: int
    ny: int
    h: tuple                  # layer thicknesses [m], surface first
    ocean_columns: int        # exact number of wet water columns
    wet_cells: int | None     # exact number of wet cells (None: as the bathymetry falls)
    wide_stencil: bool        # add the distance-2 horizontal neighbours
    seed: int = 1410


def _layers_cfg1():
    return tuple(50.0 * 10.0 ** (k / 7.0) for k in range(8))


def _layers_cfg2():
    # 50, 70, 100, 140, 190, then +50 m per layer to 690 m: 15 layers, 5200 m in total.
    return (50.0, 70.0, 100.0, 140.0, 190.0) + tuple(190.0 + 50.0 * i for i in range(1, 11))


def _layers_cfg5():
    return tuple(10.0 * 50.0 ** (k / 22.0) for k in range(23))


SPECS = {
    # 64 x 32 x 8, 30 % land: 1434 columns; 90 % of the 11472 column-layers are wet.
    "ndop_64x32x8": GridSpec("ndop_64x32x8", 64, 32, _layers_cfg1(), 1434, 10325, False),
    # 128 x 64 x 15: the paper's 2.8125 degree size, 52749 wet cells (Section 7), 4448 columns.
    "ndop_128x64x15": GridSpec("ndop_128x64x15", 128, 64, _layers_cfg2(), 4448, 52749, True),
    # 360 x 180 x 23 at about 65 % ocean.
    "npzd_360x180x23": GridSpec("npzd_360x180x23", 360, 180, _layers_cfg5(), 42120, 700000, True),
    # tiny grids for brute-force checks
    "tiny_4x3x3": GridSpec("tiny_4x3x3", 4, 3, (50.0, 80.0, 120.0), 9, 21, False),
    "tiny_6x4x4": GridSpec("tiny_6x4x4", 6, 4, (40.0, 60.0, 90.0, 130.0), 17, 52, True),
}


def spec(name: str) -> GridSpec:
    return SPECS[name]


@dataclasses.dataclass
class Problem:
    """All inputs of the TMM year map for one grid (host arrays, FP64 / int32)."""
    spec: GridSpec
    nstep: int                 # steps per model year
    dt: float                  # time step as a fraction of the year (1/nstep)
    nmonth: int
    # columns
    col_start: np.ndarray      # int32 [ncol+1]: first cell of each column (cells are column-major)
    col_i: np.ndarray          # int32 [ncol]: longitude index
    col_j: np.ndarray          # int32 [ncol]: latitude index
    lat: np.ndarray            # f64 [ncol]: latitude of the column centre [degrees]
    area: np.ndarray           # f64 [ncol]: surface area [m^2]
    # cells
    layer: np.ndarray          # int32 [n]
    h: np.ndarray              # f64 [n]: layer thickness [m]
    zc: np.ndarray             # f64 [n]: depth of the layer centre [m]
    vol: np.ndarray            # f64 [n]: cell volume [m^3]
    # explicit matrices, shared CSR pattern
    exp_rowptr: np.ndarray     # int32 [n+1]
    exp_colidx: np.ndarray     # int32 [nnz]
    exp_val: np.ndarray        # f64 [nmonth, nnz]
    # implicit matrices: one dense row-major block per column
    blk_off: np.ndarray        # int64 [ncol+1]: offset of each column's block
    imp_blk: np.ndarray        # f64 [nmonth, S_imp]

    @property
    def n(self) -> int:
        return int(self.col_start[-1])

    @property
    def ncol(self) -> int:
        return int(self.col_start.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.exp_colidx.shape[0])

    @property
    def s_imp(self) -> int:
        return int(self.blk_off[-1])

    @property
    def nlayer(self) -> np.ndarray:
        return np.diff(self.col_start).astype(np.int32)

    @property
    def lmax(self) -> int:
        return int(self.nlayer.max())

    def summary(self) -> dict:
        return {"grid": self.spec.name, "n": self.n, "ncol": self.ncol, "nnz": self.nnz,
                "S_imp": self.s_imp, "lmax": self.lmax, "nstep": self.nstep}

    # Dense forms, for brute-force checks on tiny grids only.
    def dense_exp(self, m: int) -> np.ndarray:
        a = np.zeros((self.n, self.n))
        for i in range(self.n):
            for p in range(self.exp_rowptr[i], self.exp_rowptr[i + 1]):
                a[i, self.exp_colidx[p]] = self.exp_val[m, p]
        return a

    def dense_imp(self, m: int) -> np.ndarray:
        b = np.zeros((self.n, self.n))
        for c in range(self.ncol):
            s, e = int(self.col_start[c]), int(self.col_start[c + 1])
            L = e - s
            o = int(self.blk_off[c])
            b[s:e, s:e] = self.imp_blk[m, o:o + L * L].reshape(L, L)
        return b


def _smooth(field: np.ndarray, passes: int) -> np.ndarray:
    """Binomial smoothing, periodic in longitude (axis 1), reflecting in latitude (axis 0)."""
    f = field
    for _ in range(passes):
        f = 0.25 * (np.roll(f, 1, axis=1) + 2.0 * f + np.roll(f, -1, axis=1))
        up = np.concatenate([f[:1], f[:-1]], axis=0)
        dn = np.concatenate([f[1:], f[-1:]], axis=0)
        f = 0.25 * (up + 2.0 * f + dn)
    return f


def _land_mask_and_depth(sp: GridSpec):
    nx, ny, nz = sp.nx, sp.ny, len(sp.h)
    passes = max(2, nx // 8)
    r = rng(sp.seed, "mask")
    m = _smooth(r.standard_normal((ny, nx)), passes)
    order = np.argsort(-m.ravel(), kind="stable")
    ocean = np.zeros(ny * nx, dtype=bool)
    ocean[order[:sp.ocean_columns]] = True
    ocean = ocean.reshape(ny, nx)

    # bathymetry: smooth noise plus distance from the coast (a smoothed ocean mask)
    rb = rng(sp.seed, "bathymetry")
    b = _smooth(rb.standard_normal((ny, nx)), passes) + 1.5 * _smooth(ocean.astype(np.float64), 2)
    jj, ii = np.nonzero(ocean)            # raster order: latitude outer, longitude inner
    vals = b[jj, ii]
    ncol = jj.shape[0]
    rank = np.empty(ncol)
    rank[np.argsort(vals, kind="stable")] = (np.arange(ncol) + 1.0) / ncol

    def depth(gamma):
        return np.clip(np.ceil(nz * rank ** gamma), 1, nz).astype(np.int64)

    if sp.wet_cells is None:
        L = depth(0.25)
    else:
        target = int(sp.wet_cells)
        if not (ncol <= target <= ncol * nz):
            raise ValueError("wet_cells out of range for this grid")
        lo, hi = 1e-4, 50.0
        for _ in range(200):
            mid = math.sqrt(lo * hi)
            if depth(mid).sum() > target:
                lo = mid
            else:
                hi = mid
        L = depth(hi)
        # exact adjustment, deepest-ranked columns first
        by_rank = np.argsort(-rank, kind="stable")
        diff = target - int(L.sum())
        while diff != 0:
            step = 1 if diff > 0 else -1
            moved = False
            for c in (by_rank if step > 0 else by_rank[::-1]):
                if diff == 0:
                    break
                if 1 <= L[c] + step <= nz:
                    L[c] += step
                    diff -= step
                    moved = True
            if not moved:
                raise ValueError("cannot reach wet_cells")
    return ocean, jj.astype(np.int32), ii.astype(np.int32), L.astype(np.int32)


def make_problem(name_or_spec, nstep: int = 2880, nmonth: int = 12) -> Problem:
    """Build the synthetic problem for a named workload (see ``SPECS``)."""
    sp = SPECS[name_or_spec] if isinstance(name_or_spec, str) else name_or_spec
    nx, ny = sp.nx, sp.ny
    hz = np.asarray(sp.h, dtype=np.float64)
    nz = hz.shape[0]
    dt_s = SECONDS_PER_YEAR / nstep

    ocean, col_j, col_i, L = _land_mask_and_depth(sp)
    ncol = col_j.shape[0]
    col_start = np.zeros(ncol + 1, dtype=np.int64)
    col_start[1:] = np.cumsum(L)
    n = int(col_start[-1])

    # geometry
    dlon = 2.0 * math.pi / nx
    dphi = math.pi / ny
    lat_edges = -0.5 * math.pi + dphi * np.arange(ny + 1)
    lat_c = lat_edges[:-1] + 0.5 * dphi
    area_j = EARTH_RADIUS ** 2 * dlon * (np.sin(lat_edges[1:]) - np.sin(lat_edges[:-1]))
    ztop = np.concatenate([[0.0], np.cumsum(hz)[:-1]])
    zcen = ztop + 0.5 * hz

    # cell id lookup [k, j, i]; -1 where dry
    cid = -np.ones((nz, ny, nx), dtype=np.int64)
    layer = np.empty(n, dtype=np.int32)
    cell_col = np.empty(n, dtype=np.int64)
    for c in range(ncol):
        s = col_start[c]
        cid[:L[c], col_j[c], col_i[c]] = s + np.arange(L[c])
        layer[s:s + L[c]] = np.arange(L[c])
        cell_col[s:s + L[c]] = c
    cell_h = hz[layer]
    cell_zc = zcen[layer]
    cell_area = area_j[col_j[cell_col]]
    vol = cell_area * cell_h

    # ---- undirected neighbour pairs, with a geometric conductance scale [m^3/s per (m^2/s)]
    pairs_p, pairs_q, geo, kind = [], [], [], []

    def add_horizontal(di, dj, label):
        for k in range(nz):
            a = cid[k]
            if dj >= 0:
                src = a[: ny - dj, :]
                dst = np.roll(a, -di, axis=1)[dj:, :]
                jsrc = np.arange(ny - dj)
            else:
                raise AssertionError
            ok = (src >= 0) & (dst >= 0)
            if di == 0 and dj == 0:
                continue
            jj_, ii_ = np.nonzero(ok)
            p = src[jj_, ii_]
            q = dst[jj_, ii_]
            jmid = jsrc[jj_] + 0.5 * dj
            phim = -0.5 * math.pi + dphi * (jmid + 0.5)
            dxm = EARTH_RADIUS * np.cos(phim) * dlon
            dy = EARTH_RADIUS * dphi
            dist = np.sqrt((di * dxm) ** 2 + (dj * dy) ** 2)
            # face length for face neighbours; a quarter-weight length for the others
            if label == "east":
                length = np.full(p.shape, dy)
            elif label == "north":
                length = EARTH_RADIUS * np.cos(-0.5 * math.pi + dphi * (jsrc[jj_] + 1)) * dlon
            else:
                length = 0.25 * np.minimum(dy, dxm)
            pairs_p.append(p)
            pairs_q.append(q)
            # grid-scaled diffusivity (proportional to cos^2 of latitude) keeps polar rates bounded
            geo.append(hz[k] * length / dist * np.cos(phim) ** 2)
            kind.append(np.full(p.shape, {"east": 0, "north": 1}.get(label, 2), dtype=np.int8))

    add_horizontal(1, 0, "east")
    add_horizontal(0, 1, "north")
    add_horizontal(1, 1, "diag")
    add_horizontal(-1, 1, "diag")
    if sp.wide_stencil:
        add_horizontal(2, 0, "far")
        add_horizontal(0, 2, "far")
    # vertical neighbours within a column
    vp = np.nonzero(layer[:-1] + 1 == layer[1:])[0]
    vp = vp[cell_col[vp] == cell_col[vp + 1]]
    pairs_p.append(vp)
    pairs_q.append(vp + 1)
    dzc = 0.5 * (cell_h[vp] + cell_h[vp + 1])
    geo.append(cell_area[vp] / dzc)
    kind.append(np.full(vp.shape, 3, dtype=np.int8))
    P = np.concatenate(pairs_p)
    Q = np.concatenate(pairs_q)
    G = np.concatenate(geo)
    K = np.concatenate(kind)
    if np.any(P == Q):
        raise ValueError("grid too small for this stencil")
    # on narrow grids two stencil offsets can name the same pair: keep the first
    key = np.minimum(P, Q) * n + np.maximum(P, Q)
    _, first = np.unique(key, return_index=True)
    keep = np.sort(first)
    P, Q, G, K = P[keep], Q[keep], G[keep], K[keep]
    npair = P.shape[0]

    # ---- streamfunction on cell corners per layer and month: corners (j in 0..ny, i in 0..nx-1)
    rp = rng(sp.seed, "psi")
    passes = max(2, nx // 8)
    base = _smooth(rp.standard_normal((ny + 1, nx)), passes)
    s1 = _smooth(rp.standard_normal((ny + 1, nx)), passes)
    s2 = _smooth(rp.standard_normal((ny + 1, nx)), passes)
    norm = max(np.abs(base).max(), 1e-30)
    base, s1, s2 = base / norm, s1 / norm, s2 / norm
    corner_phi = lat_edges[:, None] * np.ones((1, nx))
    taper = np.cos(corner_phi) ** 2
    depth_decay = np.exp(-zcen / 1500.0)
    psi_amp = 2.0e5  # m^2/s

    # corners touching a dry cell at layer k: corner (j, i) touches cells (j-1, i-1), (j-1, i), (j, i-1), (j, i)
    def corner_wet(k):
        w = (cid[k] >= 0)
        wp = np.zeros((ny + 2, nx), dtype=bool)
        wp[1:-1] = w
        c = wp[:-1] & wp[1:]                  # rows j-1 and j (padded)
        return c & np.roll(c, 1, axis=1)      # columns i-1 and i

    cw = [corner_wet(k) for k in range(nz)]

    # ---- diffusivities
    rk = rng(sp.seed, "kappa_h")
    kh_base = 2.0e3 * np.exp(-zcen / 2000.0)                      # m^2/s per layer
    pair_noise = np.exp(0.3 * rk.standard_normal((nmonth, npair)))
    kappa_v_exp = 2.0e-4                                          # m^2/s, explicit vertical exchange

    # ---- assemble the CSR pattern: diagonal + both directions of every pair
    rows = np.concatenate([np.arange(n), P, Q])
    cols = np.concatenate([np.arange(n), Q, P])
    order = np.lexsort((cols, rows))
    rows_s, cols_s = rows[order], cols[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows_s + 1, 1)
    rowptr = np.cumsum(rowptr)
    # position of each (row, col) entry in the sorted arrays
    pos = np.empty_like(order)
    pos[order] = np.arange(order.shape[0])
    pos_diag = pos[:n]
    pos_pq = pos[n:n + npair]          # entry (P, Q)
    pos_qp = pos[n + npair:]           # entry (Q, P)
    nnz = rows_s.shape[0]

    exp_val = np.zeros((nmonth, nnz))
    k_of_pair = layer[P]
    for m in range(nmonth):
        ph = 2.0 * math.pi * m / nmonth
        # advective transports of east (kind 0) and north (kind 1) faces, divergence-free per layer
        U = np.zeros(npair)                    # volume transport from P to Q [m^3/s]
        for k in range(nz):
            psi = psi_amp * depth_decay[k] * taper * (base + 0.5 * math.cos(ph) * s1 + 0.5 * math.sin(ph) * s2)
            psi = np.where(cw[k], psi, 0.0)
            psi[0, :] = 0.0
            psi[-1, :] = 0.0
            sel = (K == 0) & (k_of_pair == k)
            if np.any(sel):
                pc = P[sel]
                j = col_j[cell_col[pc]]
                i = col_i[cell_col[pc]]
                ie = (i + 1) % nx
                U[sel] = (psi[j + 1, ie] - psi[j, ie]) * hz[k]
            sel = (K == 1) & (k_of_pair == k)
            if np.any(sel):
                pc = P[sel]
                j = col_j[cell_col[pc]]
                i = col_i[cell_col[pc]]
                ie = (i + 1) % nx
                U[sel] = -(psi[j + 1, ie] - psi[j + 1, i]) * hz[k]
        seasonal = 1.0 + 0.3 * math.sin(ph + 0.7)
        D = np.where(K == 3, kappa_v_exp * seasonal * G,
                     kh_base[k_of_pair] * seasonal * G) * pair_noise[m]
        # rates [1/s]: into P from Q, and into Q from P
        into_p = D + np.maximum(-U, 0.0)    # flow from Q to P when U < 0
        into_q = D + np.maximum(U, 0.0)
        out_rate = np.zeros(n)
        np.add.at(out_rate, P, into_q)      # what leaves P goes into Q
        np.add.at(out_rate, Q, into_p)
        courant = dt_s * out_rate / vol
        scale = 1.0 if courant.max() <= 0.5 else 0.5 / courant.max()
        v = exp_val[m]
        v[pos_pq] = scale * dt_s * into_p / vol[P]
        v[pos_qp] = scale * dt_s * into_q / vol[Q]
        v[pos_diag] = 1.0 - scale * courant

    # ---- implicit blocks: (I - dt K)^{-1}, K tridiagonal vertical diffusion in flux form
    rv = rng(sp.seed, "kappa_v")
    blk_off = np.zeros(ncol + 1, dtype=np.int64)
    blk_off[1:] = np.cumsum(L.astype(np.int64) ** 2)
    s_imp = int(blk_off[-1])
    imp_blk = np.zeros((nmonth, s_imp))
    log_kv = rv.uniform(math.log(1e-5), math.log(1e-2), size=(nmonth, ncol, max(nz - 1, 1)))
    dzi = 0.5 * (hz[:-1] + hz[1:])
    for m in range(nmonth):
        for Lc in np.unique(L):
            cs = np.nonzero(L == Lc)[0]
            M = np.broadcast_to(np.eye(Lc), (cs.shape[0], Lc, Lc)).copy()
            for k in range(Lc - 1):
                g = np.exp(log_kv[m, cs, k]) / dzi[k] * dt_s    # m per step
                M[:, k, k] += g / hz[k]
                M[:, k, k + 1] -= g / hz[k]
                M[:, k + 1, k + 1] += g / hz[k + 1]
                M[:, k + 1, k] -= g / hz[k + 1]
            B = np.linalg.inv(M)
            for t, c in enumerate(cs):
                o = blk_off[c]
                imp_blk[m, o:o + Lc * Lc] = B[t].ravel()

    return Problem(
        spec=sp, nstep=nstep, dt=1.0 / nstep, nmonth=nmonth,
        col_start=col_start.astype(np.int32), col_i=col_i, col_j=col_j,
        lat=np.degrees(lat_c[col_j]).astype(np.float64), area=area_j[col_j].astype(np.float64),
        layer=layer, h=cell_h, zc=cell_zc, vol=vol,
        exp_rowptr=rowptr.astype(np.int32), exp_colidx=cols_s.astype(np.int32), exp_val=exp_val,
        blk_off=blk_off, imp_blk=imp_blk,
    )


def initial_state(prob: Problem, ntracer: int = 2, values=(2.17, 1.0e-4)) -> np.ndarray:
    """Spatially constant initial state, layout [ntracer][n] (N = 2.17, DOP = 1e-4)."""
    y = np.empty((ntracer, prob.n))
    for t in range(ntracer):
        y[t] = values[t]
    return y


def random_state(prob: Problem, ntracer: int = 2, seed: int = 1410, scale=(2.17, 0.3)) -> np.ndarray:
    """A positive, spatially varying state for parity checks (layout [ntracer][n])."""
    r = rng(seed, "state")
    y = np.empty((ntracer, prob.n))
    for t in range(ntracer):
        s = scale[t] if t < len(scale) else 0.1
        y[t] = s * (0.5 + r.random(prob.n))
    return y
