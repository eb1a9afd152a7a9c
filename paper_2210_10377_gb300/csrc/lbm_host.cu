// lbm_host.cu -- host-side geometry and argument checks (see lbm_host.h).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <thread>
#include <vector>

#include "gblbm.h"
#include "lbm_host.h"

namespace gblbm {

size_t storage_bytes(int storage)
{
    switch (storage) {
    case LBM_F64: return 8;
    case LBM_F16_DEV: return 2;
    default: return 4;
    }
}

namespace {

// Solid indices in [lo, hi): eight bytes are tested at a time (masks are
// mostly fluid) and zero words skipped.  lo is a multiple of 8.
void scan_solids(const uint8_t *mask, size_t lo, size_t hi, std::vector<long long> &out)
{
    size_t i = lo;
    for (; i + 8 <= hi; i += 8) {
        uint64_t w;
        memcpy(&w, mask + i, 8);
        if (w == 0) continue;
        for (size_t k = i; k < i + 8; ++k)
            if (mask[k]) out.push_back((long long)k);
    }
    for (; i < hi; ++i)
        if (mask[i]) out.push_back((long long)i);
}

}  // namespace

std::vector<long long> solid_nodes(const uint8_t *mask, int nx, int ny)
{
    const size_t n = (size_t)nx * ny;
    std::vector<long long> out;
    unsigned nt = 1;
    if (n >= ((size_t)1 << 22)) {
        const unsigned hc = std::thread::hardware_concurrency();
        nt = hc < 2 ? 1 : (hc < 8 ? hc : 8);
    }
    if (nt > 1) {
        try {
            const size_t chunk = (n / nt + 7) & ~(size_t)7;
            std::vector<std::vector<long long>> parts(nt);
            std::vector<std::thread> th;
            for (unsigned k = 0; k < nt; ++k) {
                const size_t lo = k * chunk, hi = lo + chunk < n ? lo + chunk : n;
                if (lo < hi) th.emplace_back(scan_solids, mask, lo, hi, std::ref(parts[k]));
            }
            for (auto &t : th) t.join();
            for (auto &p : parts) out.insert(out.end(), p.begin(), p.end());
            return out;
        } catch (...) {
            out.clear();  // no threads to be had: one scan here
        }
    }
    scan_solids(mask, 0, n, out);
    return out;
}

void auto_cv(const uint8_t *mask, int nx, int ny, int periodic, int *cv, const std::vector<long long> *solids)
{
    std::vector<long long> own;
    if (!solids) {
        own = solid_nodes(mask, nx, ny);
        solids = &own;
    }
    int xmin = nx, xmax = -1, ymin = ny, ymax = -1;
    for (long long k : *solids) {
        const int x = (int)(k % nx), y = (int)(k / nx);
        xmin = x < xmin ? x : xmin;
        xmax = x > xmax ? x : xmax;
        ymin = y < ymin ? y : ymin;
        ymax = y > ymax ? y : ymax;
    }
    if (xmax < 0) {
        cv[0] = periodic ? 0 : 1;
        cv[1] = periodic ? nx - 1 : nx - 2;
        cv[2] = 0;
        cv[3] = ny - 1;
        return;
    }
    int m = (xmax - xmin + 1 + 3) / 4;
    if (m < 4) m = 4;
    int x0 = xmin - m, x1 = xmax + m, y0 = ymin - m, y1 = ymax + m;
    if (periodic) {
        if (x0 < 1 || x1 > nx - 2) {
            x0 = 0;
            x1 = nx - 1;
        }
    } else {
        x0 = x0 < 1 ? 1 : x0;
        x1 = x1 > nx - 2 ? nx - 2 : x1;
    }
    if (y0 < 1 || y1 > ny - 2) {
        y0 = 0;
        y1 = ny - 1;
    }
    cv[0] = x0;
    cv[1] = x1;
    cv[2] = y0;
    cv[3] = y1;
}

// Each link's populations f_i and f_opp carry w_i rho0 each, and so does the
// bounced ft_i.  Links are enumerated from the solid nodes, crossings from the
// box edge.
void base_sums(const uint8_t *mask, int nx, int ny, int periodic, const int *cv, double rho0,
               double *link_base, double *flux_base, const std::vector<long long> *solids)
{
    std::vector<long long> own;
    if (!solids) {
        own = solid_nodes(mask, nx, ny);
        solids = &own;
    }
    const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    auto W = [](int i) { return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); };
    auto solid = [&](int x, int y) { return mask[(size_t)y * nx + x] != 0; };
    // coordinates here are at most two nodes outside the grid
    auto wrap = [&](int &x, int &y) {
        y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
        if (x < 0 || x >= nx) {
            if (!periodic) return false;
            x = x < 0 ? x + nx : x - nx;
        }
        return true;
    };
    double lb[2] = {0, 0};
    for (long long k : *solids) {  // row-major, like a plain double loop
        const int x = (int)(k % nx), y = (int)(k / nx);
        for (int i = 1; i < 9; ++i) {  // fluid x_f = s - c_i with x_f + c_i = s
            int xf = x - CX[i], yf = y - CY[i];
            if (!wrap(xf, yf) || solid(xf, yf)) continue;
            lb[0] += CX[i] * W(i);
            lb[1] += CY[i] * W(i);
        }
    }
    double fb[2] = {0, 0};
    auto inbox = [&](int x, int y) { return x >= cv[0] && x <= cv[1] && y >= cv[2] && y <= cv[3]; };
    for (int y = cv[2] - 1; y <= cv[3] + 1; ++y)
        for (int x = cv[0] - 1; x <= cv[1] + 1; ++x) {
            if (y > cv[2] && y < cv[3] && x > cv[0] && x < cv[1]) {
                x = cv[1] - 1;  // every neighbour of an interior node is inside: no crossing
                continue;
            }
            int xn = x, yn = y;
            if (!wrap(xn, yn)) continue;
            if (x != xn || y != yn) continue;  // each node once, in unwrapped position
            if (solid(xn, yn)) continue;
            const bool in = inbox(xn, yn);
            for (int i = 1; i < 9; ++i) {
                int x2 = xn + CX[i], y2 = yn + CY[i];
                if (!wrap(x2, y2) || solid(x2, y2) || inbox(x2, y2) == in) continue;
                const double s = in ? -1.0 : 1.0;
                fb[0] += s * CX[i] * W(i);
                fb[1] += s * CY[i] * W(i);
            }
        }
    link_base[0] = 2.0 * rho0 * lb[0];
    link_base[1] = 2.0 * rho0 * lb[1];
    flux_base[0] = rho0 * fb[0];
    flux_base[1] = rho0 * fb[1];
}

bool range_ok(int lo, int hi, int n, bool whole_allowed)
{
    if (lo > hi) return false;
    if (lo >= 1 && hi <= n - 2) return true;
    return whole_allowed && lo == 0 && hi == n - 1;
}

bool finite_all(const double *v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

std::string check_domain(const uint8_t *mask, int nx, int ny, double tau, const double *u_in,
                         int n_u_in, int periodic, const int *cv_in, int *cv_out,
                         const std::vector<long long> *solids)
{
    char buf[256];
    if (!mask || !u_in) return "mask and u_in must not be NULL";
    if (nx < 4 || ny < 3) {
        snprintf(buf, sizeof(buf), "grid %dx%d too small (nx >= 4, ny >= 3)", nx, ny);
        return buf;
    }
    if ((long long)nx * ny * 8 >= (1LL << 31)) {
        snprintf(buf, sizeof(buf), "grid %dx%d too large for int32 link indices", nx, ny);
        return buf;
    }
    if (!(tau > 0.5) || !std::isfinite(tau)) {
        snprintf(buf, sizeof(buf), "tau must be finite and > 0.5 (got %g)", tau);
        return buf;
    }
    if (n_u_in != 1 && n_u_in != ny) {
        snprintf(buf, sizeof(buf), "n_u_in must be 1 or ny (got %d)", n_u_in);
        return buf;
    }
    if (!finite_all(u_in, n_u_in)) return "u_in is not finite";
    if (!periodic) {
        const int cols[4] = {0, 1, nx - 2, nx - 1};
        for (int y = 0; y < ny; ++y)
            for (int c : cols)
                if (mask[(size_t)y * nx + c]) {
                    snprintf(buf, sizeof(buf),
                             "solid node at (%d, %d): columns 0, 1, nx-2, nx-1 of a channel must be fluid",
                             c, y);
                    return buf;
                }
    }
    int cv[4];
    if (!cv_in || cv_in[0] < 0) {
        auto_cv(mask, nx, ny, periodic, cv, solids);
    } else {
        memcpy(cv, cv_in, sizeof(cv));
        if (!range_ok(cv[0], cv[1], nx, periodic != 0) || !range_ok(cv[2], cv[3], ny, true)) {
            snprintf(buf, sizeof(buf),
                     "control volume {%d,%d,%d,%d} must lie within [1, n-2] (or span a periodic direction)",
                     cv[0], cv[1], cv[2], cv[3]);
            return buf;
        }
    }
    memcpy(cv_out, cv, sizeof(cv));
    return std::string();
}

void cv_tile_rect(const int *cv, int nx, int ny, int tw, int th, int *cvt)
{
    const int hx0 = cv[0] - 1 < 0 ? 0 : cv[0] - 1, hx1 = cv[1] + 1 > nx - 1 ? nx - 1 : cv[1] + 1;
    const int hy0 = cv[2] - 1 < 0 ? 0 : cv[2] - 1, hy1 = cv[3] + 1 > ny - 1 ? ny - 1 : cv[3] + 1;
    cvt[0] = hx0 / tw;
    cvt[1] = hx1 / tw;
    cvt[2] = hy0 / th;
    cvt[3] = hy1 / th;
}

}  // namespace gblbm
