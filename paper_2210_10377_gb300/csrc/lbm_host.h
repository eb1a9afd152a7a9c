// lbm_host.h -- host-side geometry and argument checks shared by the
// single-domain handle (lbm_api.cu) and the batch handle (lbm_batch_api.cu).
// Plain C++ on host data; no device work.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace gblbm {

size_t storage_bytes(int storage);

bool finite_all(const double *v, int n);

// [lo, hi] lies inside [1, n-2], or spans [0, n-1] when whole_allowed.
bool range_ok(int lo, int hi, int n, bool whole_allowed);

// Row-major indices of the solid (nonzero) mask bytes.  Large masks are
// scanned by a few host threads over row ranges; the order is the same.
std::vector<long long> solid_nodes(const uint8_t *mask, int nx, int ny);

// The functions below that scan the mask take its solid nodes instead when
// given (solids: solid_nodes of the same mask), so that a caller scans once.

// Default control volume (Eq. rtt7's box V): the solid nodes' bounding box
// widened by max(4, ceil(w/4)) nodes per side, w its width in x; clipped to
// [1, nx-2] in x for a channel; a range that would reach a periodic edge
// becomes the whole period.  No solid node: the whole fluid domain.
void auto_cv(const uint8_t *mask, int nx, int ny, int periodic, int *cv,
             const std::vector<long long> *solids = nullptr);

// Momentum of the deviation base w_i rho0 over the fluid-solid links
// (link_base = 2 rho0 sum c_i w_i) and over the box-surface crossings
// (flux_base = rho0 sum of +-c_i w_i, + entering); geometry only.
void base_sums(const uint8_t *mask, int nx, int ny, int periodic, const int *cv, double rho0,
               double *link_base, double *flux_base, const std::vector<long long> *solids = nullptr);

// Checks one domain's arguments: grid size, tau, inlet profile, the fluid
// columns 0, 1, nx-2, nx-1 of a channel, and the control volume (cv_in[0] < 0
// selects the default).  On success cv_out holds the box and the result is
// empty; otherwise it is the reason.
std::string check_domain(const uint8_t *mask, int nx, int ny, double tau, const double *u_in,
                         int n_u_in, int periodic, const int *cv_in, int *cv_out,
                         const std::vector<long long> *solids = nullptr);

// Tile rectangle [tx0, tx1] x [ty0, ty1] (inclusive, in tiles of tw x th
// nodes) holding the control volume and its one-node halo, clipped to the grid.
void cv_tile_rect(const int *cv, int nx, int ny, int tw, int th, int *cvt);

}  // namespace gblbm
