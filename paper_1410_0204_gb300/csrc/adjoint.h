// adjoint.h -- set-up of the adjoint year map (internal).
#pragma once

#include <algorithm>
#include <vector>

#include "context.h"

// Host-side layouts built by metos3d_init that the adjoint set-up reuses.
struct AdjointSetup {
    const m3d_grid *g;
    const m3d_matrices *mt;
    long long s_imp;
    const std::vector<int> *sp_rows_flat, *sp_len, *sp_off;
    const std::vector<int> *bk_rows_flat, *bk_len, *bk_off;
    const std::vector<int> *bounds, *cell_col;
    const std::vector<long long> *blk_off;
};

// Build the transposed operators and tables of the adjoint (no-op where it does not apply).
m3d_status setup_adjoint(m3d_ctx *c, const AdjointSetup &in);

// Thomas factors of M when the row-major L x L block B is the inverse of a tridiagonal M.
bool tridiagonal_factors(const double *B, int L, double *nl, double *rd, double *ne);
