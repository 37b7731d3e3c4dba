// Symbolic phase of the local solver: geometric nested dissection of one slab shape.
//
// The paper performs the local solves with a supernodal multifrontal solver on a
// nested-dissection ordering ("Local Solves: Parallel Multi-frontal Methods" section:
// reorder to reduce fill, multifrontal factorization, forward/backward substitution;
// Complexity section: O(alpha n) unknowns in the biggest front of a quasi-2D layer).
// Here the ordering is purely geometric: the slab box is bisected recursively along its
// longest side by a one-cell-thick plane (the separator), down to leaf boxes of at most
// `leaf` cells.  Every tree node owns its separator (or leaf box); its update set is
// the one-cell shell of its subtree box (the face neighbours outside the box), which is
// exactly the set of ancestor-separator unknowns coupled to the subtree after
// elimination for a 7-point stencil.
#include <algorithm>
#include <cassert>
#include <functional>
#include <stdexcept>

#include "hz_internal.cuh"

namespace hz {

namespace {

struct Box { int x0, x1, y0, y1, z0, z1; };

inline long long box_vol(const Box& b) {
    return (long long)(b.x1 - b.x0) * (b.y1 - b.y0) * (b.z1 - b.z0);
}

}  // namespace

void build_shape(Shape& s, int nx, int ny, int nz, int leaf) {
    s.nx = nx; s.ny = ny; s.nz = nz;
    s.N = (long long)nx * ny * nz;
    s.nodes.clear();
    s.perm.clear();
    s.perm.reserve(s.N);

    auto cell = [&](int x, int y, int z) { return (z * ny + y) * nx + x; };

    // --- recursive bisection; nodes are pushed in post-order (children first) ---
    std::function<int(Box)> rec = [&](Box b) -> int {
        int dims[3] = {b.x1 - b.x0, b.y1 - b.y0, b.z1 - b.z0};
        int dmax = std::max(dims[0], std::max(dims[1], dims[2]));
        Node nd;
        nd.box[0] = b.x0; nd.box[1] = b.x1; nd.box[2] = b.y0; nd.box[3] = b.y1;
        nd.box[4] = b.z0; nd.box[5] = b.z1;
        Box own = b;
        if (!(box_vol(b) <= leaf || dmax < 3)) {
            int a = (dims[0] >= dims[1] && dims[0] >= dims[2]) ? 0 : (dims[1] >= dims[2] ? 1 : 2);
            Box b1 = b, b2 = b;
            int lo = a == 0 ? b.x0 : (a == 1 ? b.y0 : b.z0);
            int hi = a == 0 ? b.x1 : (a == 1 ? b.y1 : b.z1);
            int mid = (lo + hi) / 2;
            if (a == 0) { b1.x1 = mid; b2.x0 = mid + 1; own.x0 = mid; own.x1 = mid + 1; }
            if (a == 1) { b1.y1 = mid; b2.y0 = mid + 1; own.y0 = mid; own.y1 = mid + 1; }
            if (a == 2) { b1.z1 = mid; b2.z0 = mid + 1; own.z0 = mid; own.z1 = mid + 1; }
            int c1 = rec(b1);
            int c2 = rec(b2);
            nd.child[0] = c1; nd.child[1] = c2; nd.nchild = 2;
        }
        nd.sep[0] = own.x0; nd.sep[1] = own.x1; nd.sep[2] = own.y0; nd.sep[3] = own.y1;
        nd.sep[4] = own.z0; nd.sep[5] = own.z1;
        nd.own0 = (int)s.perm.size();
        for (int z = own.z0; z < own.z1; ++z)
            for (int y = own.y0; y < own.y1; ++y)
                for (int x = own.x0; x < own.x1; ++x) s.perm.push_back(cell(x, y, z));
        nd.nown = (int)s.perm.size() - nd.own0;
        int id = (int)s.nodes.size();
        s.nodes.push_back(nd);
        for (int k = 0; k < s.nodes[id].nchild; ++k) s.nodes[s.nodes[id].child[k]].parent = id;
        return id;
    };
    rec(Box{0, nx, 0, ny, 0, nz});
    if ((long long)s.perm.size() != s.N) throw Error{HZ_ERR_ARG, "nested dissection lost cells"};

    s.pos.assign(s.N, -1);
    for (long long e = 0; e < s.N; ++e) s.pos[s.perm[e]] = (int)e;

    // --- heights ---
    int H = 0;
    for (auto& nd : s.nodes) {
        int h = 0;
        for (int k = 0; k < nd.nchild; ++k) h = std::max(h, s.nodes[nd.child[k]].height + 1);
        nd.height = h;
        H = std::max(H, h);
    }
    s.levels.assign(H + 1, {});
    for (int i = 0; i < (int)s.nodes.size(); ++i) s.levels[s.nodes[i].height].push_back(i);

    // --- update sets: the face shell of the subtree box, in elimination order ---
    s.upd_idx.clear();
    std::vector<int> tmp;
    for (auto& nd : s.nodes) {
        tmp.clear();
        int x0 = nd.box[0], x1 = nd.box[1], y0 = nd.box[2], y1 = nd.box[3], z0 = nd.box[4], z1 = nd.box[5];
        auto face = [&](int ax0, int ax1, int ay0, int ay1, int az0, int az1) {
            for (int z = az0; z < az1; ++z)
                for (int y = ay0; y < ay1; ++y)
                    for (int x = ax0; x < ax1; ++x) tmp.push_back(s.pos[cell(x, y, z)]);
        };
        if (x0 > 0) face(x0 - 1, x0, y0, y1, z0, z1);
        if (x1 < nx) face(x1, x1 + 1, y0, y1, z0, z1);
        if (y0 > 0) face(x0, x1, y0 - 1, y0, z0, z1);
        if (y1 < ny) face(x0, x1, y1, y1 + 1, z0, z1);
        if (z0 > 0) face(x0, x1, y0, y1, z0 - 1, z0);
        if (z1 < nz) face(x0, x1, y0, y1, z1, z1 + 1);
        std::sort(tmp.begin(), tmp.end());
        nd.upd_off = (long long)s.upd_idx.size();
        nd.nupd = (int)tmp.size();
        s.upd_idx.insert(s.upd_idx.end(), tmp.begin(), tmp.end());
    }

    // --- front and factor-storage offsets, flop counts ---
    s.front_total = 0;
    s.factor_tiles = 0;
    s.factor_flops = 0;
    s.solve_flops_per_col = 0;
    s.max_m = 0;
    for (auto& nd : s.nodes) {
        nd.m = nd.nown + nd.nupd;
        s.max_m = std::max(s.max_m, nd.m);
        nd.front_off = s.front_total;
        s.front_total += (long long)nd.m * nd.m;
        nd.own_t = cdiv(nd.nown, TILE);
        nd.upd_t = cdiv(nd.nupd, TILE);
        nd.linv_off = s.factor_tiles;
        s.factor_tiles += (long long)nd.own_t * (nd.own_t + 1) / 2;
        nd.l21_off = s.factor_tiles;
        s.factor_tiles += (long long)nd.upd_t * nd.own_t;
        double o = nd.nown, u = nd.nupd;
        // complex multiply-adds (8 real flops each): pivot LDL^T o^3/6, its inverse o^3/6,
        // panel solve u o^2/2, Schur update u^2 o/2
        s.factor_flops += 8.0 * (o * o * o / 3.0 + u * o * o / 2.0 + u * u * o / 2.0);
        // substitution: L^{-1} and L^{-T} (o^2/2 each) + L21 and L21^T (u o each)
        s.solve_flops_per_col += 8.0 * (o * o + 2.0 * u * o);
    }

    // --- assembly map: original lower-triangle entries of every front's own columns ---
    s.asm_entries.clear();
    const int ddx[7] = {0, -1, 1, 0, 0, 0, 0};
    const int ddy[7] = {0, 0, 0, -1, 1, 0, 0};
    const int ddz[7] = {0, 0, 0, 0, 0, -1, 1};
    for (auto& nd : s.nodes) {
        nd.asm_off = (long long)s.asm_entries.size();
        const int* ub = s.upd_idx.data() + nd.upd_off;
        for (int pc = 0; pc < nd.nown; ++pc) {
            int e = nd.own0 + pc;
            int c = s.perm[e];
            int x = c % nx, y = (c / nx) % ny, z = c / (nx * ny);
            for (int d = 0; d < 7; ++d) {
                int qx = x + ddx[d], qy = y + ddy[d], qz = z + ddz[d];
                if (qx < 0 || qx >= nx || qy < 0 || qy >= ny || qz < 0 || qz >= nz) continue;
                int eq = s.pos[cell(qx, qy, qz)];
                if (eq < e) continue;  // upper triangle: assembled in a descendant's front
                int row;
                if (eq < nd.own0 + nd.nown) {
                    row = eq - nd.own0;
                } else {
                    const int* it = std::lower_bound(ub, ub + nd.nupd, eq);
                    if (it == ub + nd.nupd || *it != eq)
                        throw Error{HZ_ERR_ARG, "symbolic: coupled unknown missing from update set"};
                    row = nd.nown + (int)(it - ub);
                }
                AsmEntry a;
                a.foff = (long long)row + (long long)pc * nd.m;
                a.cell = c;
                a.dir = d;
                s.asm_entries.push_back(a);
            }
        }
        nd.nasm = (int)((long long)s.asm_entries.size() - nd.asm_off);
    }

    // --- extend-add maps: child update unknown -> parent front position ---
    s.emap.clear();
    for (auto& nd : s.nodes) {
        nd.emap_off = (long long)s.emap.size();
        if (nd.parent < 0) {
            if (nd.nupd != 0) throw Error{HZ_ERR_ARG, "symbolic: root with a non-empty update set"};
            continue;
        }
        const Node& p = s.nodes[nd.parent];
        const int* ub = s.upd_idx.data() + nd.upd_off;
        const int* pb = s.upd_idx.data() + p.upd_off;
        for (int a = 0; a < nd.nupd; ++a) {
            int e = ub[a];
            int posn;
            if (e >= p.own0 && e < p.own0 + p.nown) {
                posn = e - p.own0;
            } else {
                const int* it = std::lower_bound(pb, pb + p.nupd, e);
                if (it == pb + p.nupd || *it != e)
                    throw Error{HZ_ERR_ARG, "symbolic: child update unknown not in parent front"};
                posn = p.nown + (int)(it - pb);
            }
            s.emap.push_back(posn);
        }
    }
}

}  // namespace hz
