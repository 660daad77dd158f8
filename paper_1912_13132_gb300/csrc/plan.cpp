// plan.cpp -- subset membership (Sec. 2.3 of arXiv 1912.13132) on the host.
//
// The domain D is cut into disjoint cores D_i; subset i trains on the TRAIN points
// inside D_i and its shell of width delta (Eq. 5-6, Fig. 1) and validates on the
// VALID points inside D_i.  Readings fixed by the ABI (include/pcv.h):
// half-open cores closed on D's upper edges, closed L-infinity windows
// [x0 - delta, x1 + delta] x [y0 - delta, y1 + delta], ascending index order.
//
// Regular layouts are built in O(n + sum_i k_i): each point finds the range of
// windows that can hold it by binary search on the (monotone) window edges and
// is appended to those subsets, points visited in ascending order.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "pcv_internal.h"

namespace pcv {

namespace {

std::vector<double> cut_points(double lo, double hi, int n) {
    std::vector<double> b(n + 1);
    for (int c = 0; c <= n; ++c) b[c] = lo + ((hi - lo) * (double)c) / (double)n;
    b[0] = lo;
    b[n] = hi;
    return b;
}

// Largest c in [0, n) such that point coordinate x lies in core c of the cut
// points b (half-open, the last cell closed); -1 when outside [b[0], b[n]].
int core_index(const std::vector<double>& b, double x) {
    int n = (int)b.size() - 1;
    if (!(x >= b[0]) || !(x <= b[n])) return -1;
    int c = (int)(std::upper_bound(b.begin(), b.end(), x) - b.begin()) - 1;
    if (c >= n) c = n - 1;  // x == b[n]: closed upper edge
    return c;
}

}  // namespace

pcv_status build_plan(const double* xy, const uint8_t* role, int64_t n, const pcv_layout* L,
                      Plan& P, std::string& err) {
    if (n < 0) { err = "n < 0"; return PCV_ERR_ARG; }
    if (n > 0 && (!xy || !role)) { err = "NULL xy or role"; return PCV_ERR_ARG; }
    if (!L) { err = "NULL layout"; return PCV_ERR_ARG; }
    if (!(L->delta >= 0.0) || !std::isfinite(L->delta)) { err = "delta must be finite and >= 0"; return PCV_ERR_ARG; }
    if (n > INT32_MAX) { err = "n exceeds 2^31 - 1"; return PCV_ERR_ARG; }
    for (int64_t j = 0; j < n; ++j) {
        if (role[j] > PCV_ROLE_IGNORE) { err = "role out of range"; return PCV_ERR_ARG; }
        if (!std::isfinite(xy[2 * j]) || !std::isfinite(xy[2 * j + 1])) { err = "non-finite coordinate"; return PCV_ERR_ARG; }
    }
    pcv_rect D;
    if (L->has_domain) {
        D = L->domain;
    } else {
        if (n == 0) { err = "empty input needs an explicit domain"; return PCV_ERR_ARG; }
        D = {xy[0], xy[0], xy[1], xy[1]};
        for (int64_t j = 1; j < n; ++j) {
            D.x0 = std::min(D.x0, xy[2 * j]);
            D.x1 = std::max(D.x1, xy[2 * j]);
            D.y0 = std::min(D.y0, xy[2 * j + 1]);
            D.y1 = std::max(D.y1, xy[2 * j + 1]);
        }
    }
    if (!std::isfinite(D.x0) || !std::isfinite(D.x1) || !std::isfinite(D.y0) || !std::isfinite(D.y1) ||
        !(D.x1 >= D.x0) || !(D.y1 >= D.y0)) {
        err = "invalid domain";
        return PCV_ERR_ARG;
    }
    const double d = L->delta;
    P.n = n;
    P.domain = D;
    P.delta = d;

    if (L->kind == PCV_LAYOUT_GRID) {
        if (L->nx < 1 || L->ny < 1 || (int64_t)L->nx * L->ny > (1 << 24)) { err = "bad nx/ny"; return PCV_ERR_ARG; }
        const int nx = L->nx, ny = L->ny;
        const int N = nx * ny;
        auto bx = cut_points(D.x0, D.x1, nx), by = cut_points(D.y0, D.y1, ny);
        // window edges: lo[c] = b[c] - delta, hi[c] = b[c+1] + delta (both nondecreasing in c)
        std::vector<double> wxl(nx), wxh(nx), wyl(ny), wyh(ny);
        for (int c = 0; c < nx; ++c) { wxl[c] = bx[c] - d; wxh[c] = bx[c + 1] + d; }
        for (int c = 0; c < ny; ++c) { wyl[c] = by[c] - d; wyh[c] = by[c + 1] + d; }
        P.N = N;
        P.cores.resize(N);
        for (int cy = 0; cy < ny; ++cy)
            for (int cx = 0; cx < nx; ++cx) P.cores[cy * nx + cx] = {bx[cx], bx[cx + 1], by[cy], by[cy + 1]};
        // window range of coordinate x: cells c with lo[c] <= x <= hi[c]
        auto wrange = [](const std::vector<double>& lo, const std::vector<double>& hi, double x, int& a, int& b) {
            a = (int)(std::lower_bound(hi.begin(), hi.end(), x) - hi.begin());        // first hi >= x
            b = (int)(std::upper_bound(lo.begin(), lo.end(), x) - lo.begin()) - 1;    // last lo <= x
        };
        std::vector<int64_t> tcnt(N + 1, 0), vcnt(N + 1, 0);
        for (int pass = 0; pass < 2; ++pass) {
            std::vector<int64_t> tpos, vpos;
            if (pass == 1) {
                P.T_off.assign(N + 1, 0);
                P.V_off.assign(N + 1, 0);
                for (int i = 0; i < N; ++i) { P.T_off[i + 1] = P.T_off[i] + tcnt[i]; P.V_off[i + 1] = P.V_off[i] + vcnt[i]; }
                P.T_idx.resize(P.T_off[N]);
                P.V_idx.resize(P.V_off[N]);
                tpos.assign(P.T_off.begin(), P.T_off.end() - 1);
                vpos.assign(P.V_off.begin(), P.V_off.end() - 1);
            }
            for (int64_t j = 0; j < n; ++j) {
                const double x = xy[2 * j], y = xy[2 * j + 1];
                if (role[j] == PCV_ROLE_TRAIN) {
                    int ax, bxx, ay, byy;
                    wrange(wxl, wxh, x, ax, bxx);
                    wrange(wyl, wyh, y, ay, byy);
                    for (int cy = ay; cy <= byy; ++cy)
                        for (int cx = ax; cx <= bxx; ++cx) {
                            // the binary searches give the exact set; the test below restates it
                            if (!(wxl[cx] <= x && x <= wxh[cx] && wyl[cy] <= y && y <= wyh[cy])) continue;
                            int i = cy * nx + cx;
                            if (pass == 0) ++tcnt[i]; else P.T_idx[tpos[i]++] = j;
                        }
                } else if (role[j] == PCV_ROLE_VALID) {
                    int cx = core_index(bx, x), cy = core_index(by, y);
                    if (cx < 0 || cy < 0) continue;
                    int i = cy * nx + cx;
                    if (pass == 0) ++vcnt[i]; else P.V_idx[vpos[i]++] = j;
                }
            }
        }
        return PCV_OK;
    }
    if (L->kind == PCV_LAYOUT_RECTS) {
        if (L->n_cores < 1 || !L->cores) { err = "rects layout needs cores"; return PCV_ERR_ARG; }
        const int N = L->n_cores;
        P.N = N;
        P.cores.assign(L->cores, L->cores + N);
        for (const auto& r : P.cores)
            if (!std::isfinite(r.x0) || !std::isfinite(r.x1) || !std::isfinite(r.y0) || !std::isfinite(r.y1) ||
                !(r.x1 >= r.x0) || !(r.y1 >= r.y0)) { err = "invalid core rectangle"; return PCV_ERR_ARG; }
        P.T_off.assign(N + 1, 0);
        P.V_off.assign(N + 1, 0);
        P.T_idx.clear();
        P.V_idx.clear();
        for (int i = 0; i < N; ++i) {
            const pcv_rect r = P.cores[i];
            const bool xc = (r.x1 == D.x1), yc = (r.y1 == D.y1);
            const double wx0 = r.x0 - d, wx1 = r.x1 + d, wy0 = r.y0 - d, wy1 = r.y1 + d;
            for (int64_t j = 0; j < n; ++j) {
                const double x = xy[2 * j], y = xy[2 * j + 1];
                if (role[j] == PCV_ROLE_TRAIN && wx0 <= x && x <= wx1 && wy0 <= y && y <= wy1) P.T_idx.push_back(j);
            }
            for (int64_t j = 0; j < n; ++j) {
                const double x = xy[2 * j], y = xy[2 * j + 1];
                if (role[j] != PCV_ROLE_VALID) continue;
                if (!(x >= r.x0) || !(xc ? x <= r.x1 : x < r.x1)) continue;
                if (!(y >= r.y0) || !(yc ? y <= r.y1 : y < r.y1)) continue;
                P.V_idx.push_back(j);
            }
            P.T_off[i + 1] = (int64_t)P.T_idx.size();
            P.V_off[i + 1] = (int64_t)P.V_idx.size();
        }
        return PCV_OK;
    }
    err = "unknown layout kind";
    return PCV_ERR_ARG;
}

}  // namespace pcv
