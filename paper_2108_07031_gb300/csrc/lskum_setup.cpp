// Host-side set-up of a point cloud for the device kernels (lskum_create).
//
//  1. Validation of the caller's cloud: sizes, flags, unit normals, CSR
//     offsets, neighbour indices (range, self, repeats, at most 20).
//  2. Point order on the device: a Hilbert space-filling curve over the
//     cloud's bounding box, so that the 32 points of a warp and their
//     stencils are close in memory and neighbour gathers hit L1/L2.
//  3. Per neighbour slot, the split-stencil membership of Eq. 14 (decided
//     in FP64 from the sign of ds = (x_j - x_i) t_x + (y_j - y_i) t_y and of
//     dn, with t = (n_y, -n_x), n the local frame at wall/outer points and
//     the global frame at interior points), and the least-squares weights:
//       full stencil (Eq. 11):   q_x = sum_j wx_j dq_j,  q_y = sum_j wy_j dq_j
//       split stencil (Eq. 24):  dG/ds = sum_j ws_j dG_j, dG/dn = sum_j wn_j dG_j
//     i.e. the rows of the 2x2 inverse applied to (dx_j, dy_j), so the device
//     never forms or inverts the 2x2 matrices; the specular wall's factor on
//     dGn-/dn is folded into wn. For the FP64 inner sweeps also the products
//     wx hdx, wx hdy, wy hdx, wy hdy per slot and their sums per point.
//  4. Wall loops and their n_i ds_i for the force integral.
//
// Compiled with -ffp-contract=off: the stencil-membership signs must be the
// exact FP64 values of the products and sums above.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <sstream>

#include "lskum_internal.h"

namespace lskum {

namespace {

// Hilbert-curve index of (x, y) on a 2^order x 2^order grid (the classic
// quadrant-by-quadrant construction: at each level pick the quadrant's rank
// on the curve, then rotate/reflect the coordinates into that quadrant's
// frame).
uint64_t hilbert_index(uint64_t x, uint64_t y, int order) {
    const uint64_t side = uint64_t(1) << order;
    uint64_t d = 0;
    for (uint64_t s = side >> 1; s > 0; s >>= 1) {
        const uint64_t rx = (x & s) ? 1 : 0;
        const uint64_t ry = (y & s) ? 1 : 0;
        d += s * s * ((3 * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = side - 1 - x;
                y = side - 1 - y;
            }
            std::swap(x, y);
        }
    }
    return d;
}

struct Frame {
    double tx, ty, nx, ny;
};

inline Frame frame_of(int8_t flag, const double* nrm) {
    if (flag == LSKUM_INTERIOR) return {1.0, 0.0, 0.0, 1.0};
    return {nrm[1], -nrm[0], nrm[0], nrm[1]};
}

}  // namespace

int build_layout(int64_t n, const double* xy, const double* normals, const int8_t* flags,
                 const int32_t* off, const int32_t* idx, const lskum_options& opt,
                 HostLayout& L, std::string& err) {
    std::ostringstream msg;
    if (n < 1 || n > kMaxPoints) {
        msg << "n = " << n << " outside [1, " << kMaxPoints << "]";
        err = msg.str();
        return LSKUM_ERR_INVALID_ARG;
    }
    if (!xy || !normals || !flags || !off || !idx) {
        err = "null input array";
        return LSKUM_ERR_INVALID_ARG;
    }
    if (off[0] != 0) {
        err = "nbr_offsets[0] must be 0";
        return LSKUM_ERR_BAD_CONNECTIVITY;
    }
    int max_cnt = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t c = int64_t(off[i + 1]) - off[i];
        if (c < 0 || c > LSKUM_MAX_NEIGHBOURS) {
            msg << "point " << i << " has " << c << " neighbours (allowed 0.." << LSKUM_MAX_NEIGHBOURS << ")";
            err = msg.str();
            return LSKUM_ERR_BAD_CONNECTIVITY;
        }
        max_cnt = std::max<int>(max_cnt, int(c));
        if (flags[i] < 0 || flags[i] > 2) {
            msg << "point " << i << " has flag " << int(flags[i]);
            err = msg.str();
            return LSKUM_ERR_INVALID_ARG;
        }
        if (!std::isfinite(xy[2 * i]) || !std::isfinite(xy[2 * i + 1])) {
            msg << "point " << i << " has non-finite coordinates";
            err = msg.str();
            return LSKUM_ERR_INVALID_ARG;
        }
        if (flags[i] != LSKUM_INTERIOR) {
            const double a = normals[2 * i], b = normals[2 * i + 1];
            const double len2 = a * a + b * b;
            if (!(std::fabs(len2 - 1.0) <= 1e-8)) {
                msg << "boundary point " << i << " has a normal of squared length " << len2;
                err = msg.str();
                return LSKUM_ERR_INVALID_ARG;
            }
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        for (int32_t e = off[i]; e < off[i + 1]; ++e) {
            const int32_t j = idx[e];
            if (j < 0 || j >= n || j == i) {
                msg << "point " << i << " lists neighbour " << j;
                err = msg.str();
                return LSKUM_ERR_BAD_CONNECTIVITY;
            }
            for (int32_t f = off[i]; f < e; ++f) {
                if (idx[f] == j) {
                    msg << "point " << i << " lists neighbour " << j << " twice";
                    err = msg.str();
                    return LSKUM_ERR_BAD_CONNECTIVITY;
                }
            }
        }
    }

    // ---- device order
    L.n = n;
    L.stride = (n + 31) / 32 * 32;
    L.slots = max_cnt;
    L.dev_to_user.resize(n);
    std::iota(L.dev_to_user.begin(), L.dev_to_user.end(), 0);
    if (opt.reorder) {
        double xmin = xy[0], xmax = xy[0], ymin = xy[1], ymax = xy[1];
        for (int64_t i = 1; i < n; ++i) {
            xmin = std::min(xmin, xy[2 * i]);
            xmax = std::max(xmax, xy[2 * i]);
            ymin = std::min(ymin, xy[2 * i + 1]);
            ymax = std::max(ymax, xy[2 * i + 1]);
        }
        const int order = 21;
        const double side = double((uint64_t(1) << order) - 1);
        const double span = std::max(std::max(xmax - xmin, ymax - ymin), 1e-300);
        std::vector<uint64_t> key(n);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            const uint64_t hx = uint64_t((xy[2 * i] - xmin) / span * side);
            const uint64_t hy = uint64_t((xy[2 * i + 1] - ymin) / span * side);
            key[i] = hilbert_index(hx, hy, order);
        }
        std::stable_sort(L.dev_to_user.begin(), L.dev_to_user.end(),
                         [&](int32_t a, int32_t b) { return key[a] < key[b]; });
    }
    L.user_to_dev.resize(n);
    for (int64_t d = 0; d < n; ++d) L.user_to_dev[L.dev_to_user[d]] = int32_t(d);

    // ---- per point data and slot arrays
    const int64_t S = L.stride;
    const int slots = std::max(L.slots, 1);
    L.cnt.assign(n, 0);
    L.flag.assign(n, 0);
    L.nrm.assign(2 * n, 0.0);
    L.dmin.assign(n, 0.0);
    L.nbr.assign(size_t(slots) * S, 0u);
    L.hdx.assign(size_t(slots) * S, 0.0);
    L.hdy.assign(size_t(slots) * S, 0.0);
    L.wx.assign(size_t(slots) * S, 0.0);
    L.wy.assign(size_t(slots) * S, 0.0);
    L.ws.assign(size_t(slots) * S, 0.0);
    L.wn.assign(size_t(slots) * S, 0.0);
    const bool want_lc = opt.precision == LSKUM_FP64;
    if (want_lc) {
        L.lc.assign(size_t(slots) * S * 4, 0.0);
        L.lsum.assign(size_t(n) * 4, 0.0);
    }

    int64_t bad_point = -1;
    const char* bad_what = "";
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t d = 0; d < n; ++d) {
        const int64_t i = L.dev_to_user[d];
        const int8_t fl = flags[i];
        const int c = off[i + 1] - off[i];
        L.cnt[d] = c;
        L.flag[d] = fl;
        if (fl == LSKUM_INTERIOR) {
            L.nrm[2 * d] = 0.0;
            L.nrm[2 * d + 1] = 1.0;
        } else {
            L.nrm[2 * d] = normals[2 * i];
            L.nrm[2 * d + 1] = normals[2 * i + 1];
        }
        const Frame F = frame_of(fl, normals + 2 * i);
        const bool use[4] = {true, true, fl != LSKUM_WALL, fl != LSKUM_OUTER};  // s+, s-, n+, n-
        double dx[LSKUM_MAX_NEIGHBOURS], dy[LSKUM_MAX_NEIGHBOURS], wt[LSKUM_MAX_NEIGHBOURS];
        double ds[LSKUM_MAX_NEIGHBOURS], dn[LSKUM_MAX_NEIGHBOURS];
        int sl_s[LSKUM_MAX_NEIGHBOURS], sl_n[LSKUM_MAX_NEIGHBOURS];
        double sxx = 0, sxy = 0, syy = 0;
        double sss[4] = {0, 0, 0, 0}, ssn[4] = {0, 0, 0, 0}, snn[4] = {0, 0, 0, 0};
        int members[4] = {0, 0, 0, 0};
        double dmin = INFINITY;
        for (int k = 0; k < c; ++k) {
            const int32_t j = idx[off[i] + k];
            dx[k] = xy[2 * j] - xy[2 * i];
            dy[k] = xy[2 * j + 1] - xy[2 * i + 1];
            const double d2 = dx[k] * dx[k] + dy[k] * dy[k];
            const double dist = std::sqrt(d2);
            dmin = std::min(dmin, dist);
            // least-squares weight |P_j - P_i|^-p (1 for the unweighted default)
            wt[k] = opt.weight_power == 0.0 ? 1.0 : std::pow(d2, -0.5 * opt.weight_power);
            sxx += wt[k] * dx[k] * dx[k];
            sxy += wt[k] * dx[k] * dy[k];
            syy += wt[k] * dy[k] * dy[k];
            ds[k] = dx[k] * F.tx + dy[k] * F.ty;
            dn[k] = dx[k] * F.nx + dy[k] * F.ny;
            sl_s[k] = ds[k] < 0.0 ? 0 : (ds[k] > 0.0 ? 1 : -1);
            sl_n[k] = dn[k] < 0.0 ? 2 : (dn[k] > 0.0 ? 3 : -1);
            for (int sl : {sl_s[k], sl_n[k]}) {
                if (sl < 0 || !use[sl]) continue;
                sss[sl] += wt[k] * ds[k] * ds[k];
                ssn[sl] += wt[k] * ds[k] * dn[k];
                snn[sl] += wt[k] * dn[k] * dn[k];
                members[sl] += 1;
            }
        }
        L.dmin[d] = dmin;
        const double det = sxx * syy - sxy * sxy;
        const double tr = sxx + syy;
        bool ok = c >= 2 && det > 1e-12 * tr * tr;
        const char* what = "full stencil";
        double sdet[4] = {0, 0, 0, 0};
        for (int sl = 0; sl < 4 && ok; ++sl) {
            if (!use[sl]) continue;
            sdet[sl] = sss[sl] * snn[sl] - ssn[sl] * ssn[sl];
            const double st = sss[sl] + snn[sl];
            if (members[sl] < 2 || !(sdet[sl] > 1e-12 * st * st)) {
                ok = false;
                static const char* names[4] = {"s+ split stencil (ds<0)", "s- split stencil (ds>0)",
                                               "n+ split stencil (dn<0)", "n- split stencil (dn>0)"};
                what = names[sl];
            }
        }
        if (!ok) {
#pragma omp critical
            {
                if (bad_point < 0 || i < bad_point) {
                    bad_point = i;
                    bad_what = what;
                }
            }
            continue;
        }
        const double wall_fac = (fl == LSKUM_WALL) ? opt.wall_factor : 1.0;
        for (int k = 0; k < c; ++k) {
            const int32_t j = idx[off[i] + k];
            const size_t at = size_t(k) * S + d;
            uint32_t s_code = 0, n_code = 0;
            double ws = 0.0, wn = 0.0;
            const int a = sl_s[k];
            if (a >= 0 && use[a]) {
                s_code = (a == 0) ? 1u : 2u;
                ws = wt[k] * (ds[k] * snn[a] - dn[k] * ssn[a]) / sdet[a];
            }
            const int b = sl_n[k];
            if (b >= 0 && use[b]) {
                n_code = (b == 2) ? 1u : 2u;
                wn = wt[k] * (dn[k] * sss[b] - ds[k] * ssn[b]) / sdet[b];
                if (b == 3) wn *= wall_fac;
            }
            L.nbr[at] = uint32_t(L.user_to_dev[j]) | (s_code << kIndexBits) | (n_code << (kIndexBits + 2));
            L.hdx[at] = 0.5 * dx[k];
            L.hdy[at] = 0.5 * dy[k];
            L.wx[at] = wt[k] * (dx[k] * syy - dy[k] * sxy) / det;
            L.wy[at] = wt[k] * (dy[k] * sxx - dx[k] * sxy) / det;
            L.ws[at] = ws;
            L.wn[at] = wn;
            if (want_lc) {
                double* c4 = &L.lc[4 * at];
                c4[0] = L.wx[at] * L.hdx[at];
                c4[1] = L.wx[at] * L.hdy[at];
                c4[2] = L.wy[at] * L.hdx[at];
                c4[3] = L.wy[at] * L.hdy[at];
                for (int m = 0; m < 4; ++m) L.lsum[4 * d + m] += c4[m];
            }
        }
    }
    if (bad_point >= 0) {
        msg << "point " << bad_point << ": degenerate " << bad_what;
        err = msg.str();
        return LSKUM_ERR_DEGENERATE_STENCIL;
    }

    // ---- wall loops (caller order): consecutive wall points form a loop while
    // each is a neighbour of the previous one; each loop closes on itself
    std::vector<int64_t> walls;
    for (int64_t i = 0; i < n; ++i)
        if (flags[i] == LSKUM_WALL) walls.push_back(i);
    auto is_nbr = [&](int64_t a, int64_t b) {
        for (int32_t e = off[a]; e < off[a + 1]; ++e)
            if (idx[e] == b) return true;
        for (int32_t e = off[b]; e < off[b + 1]; ++e)
            if (idx[e] == a) return true;
        return false;
    };
    L.wall_id.clear();
    L.wall_nds.clear();
    size_t start = 0;
    while (start < walls.size()) {
        size_t end = start + 1;
        while (end < walls.size() && is_nbr(walls[end - 1], walls[end])) ++end;
        const size_t m = end - start;
        for (size_t k = 0; k < m; ++k) {
            const int64_t i = walls[start + k];
            const int64_t ip = walls[start + (k + 1) % m];
            const int64_t im = walls[start + (k + m - 1) % m];
            const double ax = xy[2 * ip] - xy[2 * i], ay = xy[2 * ip + 1] - xy[2 * i + 1];
            const double bx = xy[2 * i] - xy[2 * im], by = xy[2 * i + 1] - xy[2 * im + 1];
            const double dsl = 0.5 * (std::sqrt(ax * ax + ay * ay) + std::sqrt(bx * bx + by * by));
            L.wall_id.push_back(L.user_to_dev[i]);
            L.wall_nds.push_back(normals[2 * i] * dsl);
            L.wall_nds.push_back(normals[2 * i + 1] * dsl);
        }
        start = end;
    }
    return LSKUM_OK;
}

}  // namespace lskum
