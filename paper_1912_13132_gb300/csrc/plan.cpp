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
// is appended to those subsets, points visited in ascending order.  Explicit and
// recursive cores (Sec. 2.4) search the windows' x-ranges in the points sorted by x.
// The shell cap of Sec. 4.3.2 thins over-full shells last.
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

// Core membership of a point (Sec. 2.3 reading): half-open [x0, x1) x [y0, y1), closed
// on the edges that lie on D's upper edges.
bool in_core(const pcv_rect& r, const pcv_rect& D, double x, double y) {
    const bool xc = r.x1 == D.x1, yc = r.y1 == D.y1;
    return x >= r.x0 && (xc ? x <= r.x1 : x < r.x1) && y >= r.y0 && (yc ? y <= r.y1 : y < r.y1);
}

// Membership of explicit core rectangles: each window's x-range is located by binary
// search in the points sorted by x, the candidates are tested in full and each list is
// put in ascending index order.
void rect_members(const double* xy, const uint8_t* role, int64_t n, const pcv_rect& D, double d,
                  const std::vector<pcv_rect>& cores, Plan& P) {
    const int N = (int)cores.size();
    std::vector<int64_t> order(n);
    for (int64_t j = 0; j < n; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return xy[2 * a] < xy[2 * b]; });
    std::vector<double> xs(n);
    for (int64_t p = 0; p < n; ++p) xs[p] = xy[2 * order[p]];
    P.N = N;
    P.cores = cores;
    P.T_off.assign(N + 1, 0);
    P.V_off.assign(N + 1, 0);
    P.T_idx.clear();
    P.V_idx.clear();
    std::vector<int64_t> t, v;
    for (int i = 0; i < N; ++i) {
        const pcv_rect r = cores[i];
        const double wx0 = r.x0 - d, wx1 = r.x1 + d, wy0 = r.y0 - d, wy1 = r.y1 + d;
        t.clear();
        v.clear();
        const int64_t a = std::lower_bound(xs.begin(), xs.end(), wx0) - xs.begin();
        const int64_t b = std::upper_bound(xs.begin(), xs.end(), wx1) - xs.begin();
        for (int64_t p = a; p < b; ++p) {
            const int64_t j = order[p];
            const double x = xy[2 * j], y = xy[2 * j + 1];
            if (role[j] == PCV_ROLE_TRAIN && wx0 <= x && x <= wx1 && wy0 <= y && y <= wy1) t.push_back(j);
            else if (role[j] == PCV_ROLE_VALID && in_core(r, D, x, y)) v.push_back(j);
        }
        std::sort(t.begin(), t.end());
        std::sort(v.begin(), v.end());
        P.T_idx.insert(P.T_idx.end(), t.begin(), t.end());
        P.V_idx.insert(P.V_idx.end(), v.begin(), v.end());
        P.T_off[i + 1] = (int64_t)P.T_idx.size();
        P.V_off[i + 1] = (int64_t)P.V_idx.size();
    }
}

// The recursive division of Sec. 2.4 (reading in include/pcv.h).  `win` holds every
// point inside the parent's closed window; the children's windows lie inside it.
void split_rect(const double* xy, const pcv_rect& D, double d, int q, const pcv_rect& r, int depth,
                const std::vector<int64_t>& win, std::vector<pcv_rect>& out) {
    if (depth == q) {
        out.push_back(r);
        return;
    }
    const int ax = depth % 2;                   // 0: the cut is a value of x
    const double lo = ax == 0 ? r.x0 : r.y0, hi = ax == 0 ? r.x1 : r.y1;
    std::vector<double> u;                      // coordinates of the points inside the parent
    for (int64_t j : win)
        if (in_core(r, D, xy[2 * j], xy[2 * j + 1])) u.push_back(xy[2 * j + ax]);
    std::sort(u.begin(), u.end());
    u.erase(std::unique(u.begin(), u.end()), u.end());
    double s = (lo + hi) / 2.0;
    if (u.size() >= 2) {
        std::vector<double> a;                  // axis coordinates of every point in the parent's window
        a.reserve(win.size());
        for (int64_t j : win) a.push_back(xy[2 * j + ax]);
        std::sort(a.begin(), a.end());
        int64_t best = -1;
        for (size_t m = 0; m + 1 < u.size(); ++m) {
            const double c = (u[m] + u[m + 1]) / 2.0;
            // left child's window: axis coordinate <= c + d; right child's: >= c - d
            const int64_t cl = std::upper_bound(a.begin(), a.end(), c + d) - a.begin();
            const int64_t cr = (int64_t)a.size() - (std::lower_bound(a.begin(), a.end(), c - d) - a.begin());
            const int64_t diff = cl > cr ? cl - cr : cr - cl;
            if (best < 0 || diff < best) {     // strict: ties keep the smaller cut
                best = diff;
                s = c;
            }
        }
    }
    pcv_rect left = r, right = r;
    if (ax == 0) { left.x1 = s; right.x0 = s; } else { left.y1 = s; right.y0 = s; }
    for (const pcv_rect& c : {left, right}) {
        const double wx0 = c.x0 - d, wx1 = c.x1 + d, wy0 = c.y0 - d, wy1 = c.y1 + d;
        std::vector<int64_t> cw;
        for (int64_t j : win) {
            const double x = xy[2 * j], y = xy[2 * j + 1];
            if (wx0 <= x && x <= wx1 && wy0 <= y && y <= wy1) cw.push_back(j);
        }
        split_rect(xy, D, d, q, c, depth + 1, cw, out);
    }
}

void recursive_cores(const double* xy, int64_t n, const pcv_rect& D, double d, int q, std::vector<pcv_rect>& out) {
    out.clear();
    std::vector<int64_t> win;
    for (int64_t j = 0; j < n; ++j) {
        const double x = xy[2 * j], y = xy[2 * j + 1];
        if (D.x0 - d <= x && x <= D.x1 + d && D.y0 - d <= y && y <= D.y1 + d) win.push_back(j);
    }
    split_rect(xy, D, d, q, D, 0, win, out);
}

// Output w + 1 of the SplitMix64 generator seeded with `seed` (Steele, Lea and Flood,
// "Fast splittable pseudorandom number generators", OOPSLA 2014).
uint64_t splitmix64_at(uint64_t seed, uint64_t w) {
    uint64_t z = seed + (w + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Shell cap (Sec. 4.3.2): keep `cap` of a shell's TRAIN points, the smallest keys.
void cap_shells(const double* xy, int64_t n, const pcv_rect& D, int cap, uint64_t seed, Plan& P) {
    (void)n;
    std::vector<int64_t> off(P.N + 1, 0), idx;
    idx.reserve(P.T_idx.size());
    std::vector<int64_t> core, shell;
    std::vector<std::pair<uint64_t, int64_t>> key;
    for (int i = 0; i < P.N; ++i) {
        core.clear();
        shell.clear();
        for (int64_t p = P.T_off[i]; p < P.T_off[i + 1]; ++p) {
            const int64_t j = P.T_idx[p];
            (in_core(P.cores[i], D, xy[2 * j], xy[2 * j + 1]) ? core : shell).push_back(j);
        }
        if ((int64_t)shell.size() > cap) {
            key.clear();
            for (int64_t j : shell) key.push_back({splitmix64_at(seed, ((uint64_t)i << 40) | (uint64_t)j), j});
            std::nth_element(key.begin(), key.begin() + cap, key.end());
            shell.clear();
            for (int c = 0; c < cap; ++c) shell.push_back(key[c].second);
            std::vector<int64_t> all(core);
            all.insert(all.end(), shell.begin(), shell.end());
            std::sort(all.begin(), all.end());
            idx.insert(idx.end(), all.begin(), all.end());
        } else {
            idx.insert(idx.end(), P.T_idx.begin() + P.T_off[i], P.T_idx.begin() + P.T_off[i + 1]);
        }
        off[i + 1] = (int64_t)idx.size();
    }
    P.T_idx.swap(idx);
    P.T_off.swap(off);
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
        P.nx = nx;
        P.ny = ny;
        P.bx = bx;
        P.by = by;
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
    }
    if (L->kind == PCV_LAYOUT_RECTS || L->kind == PCV_LAYOUT_RECURSIVE) {
        std::vector<pcv_rect> cores;
        if (L->kind == PCV_LAYOUT_RECTS) {
            if (L->n_cores < 1 || !L->cores) { err = "rects layout needs cores"; return PCV_ERR_ARG; }
            cores.assign(L->cores, L->cores + L->n_cores);
            for (const auto& r : cores)
                if (!std::isfinite(r.x0) || !std::isfinite(r.x1) || !std::isfinite(r.y0) || !std::isfinite(r.y1) ||
                    !(r.x1 >= r.x0) || !(r.y1 >= r.y0)) { err = "invalid core rectangle"; return PCV_ERR_ARG; }
        } else {
            if (L->q < 0 || L->q > 20) { err = "recursive layout needs 0 <= q <= 20"; return PCV_ERR_ARG; }
            recursive_cores(xy, n, D, d, L->q, cores);
        }
        rect_members(xy, role, n, D, d, cores, P);
    }
    if (L->kind == PCV_LAYOUT_GRID || L->kind == PCV_LAYOUT_RECTS || L->kind == PCV_LAYOUT_RECURSIVE) {
        if (L->shell_cap < 0) { err = "shell_cap < 0"; return PCV_ERR_ARG; }
        if (L->shell_cap > 0) cap_shells(xy, n, D, L->shell_cap, L->cap_seed, P);
        return PCV_OK;
    }
    err = "unknown layout kind";
    return PCV_ERR_ARG;
}

}  // namespace pcv
