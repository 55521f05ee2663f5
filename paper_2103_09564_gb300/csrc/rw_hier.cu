// C ABI of librw.so (declared in include/rw_api.h), second part: the LOD
// pyramid and the hierarchical tree (Sec. IV, Fig. 3 processing scheme, level
// by level), incremental passes and multi-class labels.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "rw_host.h"
#include "rw_internal.h"

using namespace rwk;
using namespace rwh;

struct rw_pyramid {
    int K = 0;                               // leaf level index
    int s = 32;
    std::vector<std::array<int, 3>> dims;    // level 0 (root) .. K (leaf), x/y/z
    uint16_t* leaf = nullptr;                // unorm16 leaf (device address)
    std::vector<float*> lv;                  // FP32 levels 0..K-1 (lv[K] = nullptr)
    int device = 0;
    int leaf_host = 0;                       // leaf level in mapped host memory
    void* leaf_host_ptr = nullptr;           // its host allocation
    int host_all = 0;                        // every level in mapped host memory
    std::vector<void*> lv_host;              // host allocations of the coarse levels (host_all)
};

namespace {

// Level storage: HBM, or pinned host memory mapped into the device's address
// space (the out-of-core placement of the leaf level).
cudaError_t level_alloc(bool host, size_t bytes, void** dev, void** host_ptr) {
    *dev = nullptr;
    *host_ptr = nullptr;
    if (!host) return cudaMalloc(dev, bytes);
    cudaError_t e = cudaHostAlloc(host_ptr, bytes, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e != cudaSuccess) return e;
    e = cudaHostGetDevicePointer(dev, *host_ptr, 0);
    if (e != cudaSuccess) {
        cudaFreeHost(*host_ptr);
        *host_ptr = nullptr;
    }
    return e;
}

void level_free(void* dev, void* host_ptr) {
    if (host_ptr) cudaFreeHost(host_ptr);
    else if (dev) cudaFree(dev);
}

}  // namespace

namespace {

struct TreeLevel {
    int nbx = 1, nby = 1, nbz = 1;
    int64_t nb = 1;
    float* P = nullptr;      // filled field (device address)
    void* P_host = nullptr;  // host allocation when the level lives in host memory
    std::vector<int32_t> flags;
    std::vector<float> mn, mx, md;
    std::vector<uint8_t> status;  // 0 absent, 1 solved (new values), 2 reused (old values)
    std::vector<uint8_t> filled;  // 1: the values came from the level fill in the last pass
    std::vector<uint8_t> changed; // 1: the values changed in the last pass
};

}  // namespace

struct rw_tree {
    const rw_pyramid* pyr = nullptr;
    rw_opts opts;
    std::vector<TreeLevel> L;
    std::vector<double> lab_xyz;
    std::vector<float> lab_val;
    std::vector<uint8_t> lab_added;
    std::vector<int32_t> lab_cls;  // class of each label, -1 when not given
    int refined = 0;         // levels of the current pass done
    int update = 0;          // current pass is incremental
    std::vector<std::array<int, 3>> resolve, reused;  // node lists for the next level
    // a level refined in parts (rw_refine_level_nodes .. rw_refine_level_finish):
    // its node lists and labels, and which of its nodes are present (solved
    // here or imported)
    int open_level = -1;
    std::vector<std::array<int, 3>> open_nodes, open_reuse;
    std::vector<rwk::LabelVox> open_labs;
    std::vector<uint8_t> open_have;
};

namespace {

struct LabelKey {
    float value;
    int conflict;
    int added;
    int32_t cls;
};

void rasterize(const rw_tree* t, int k, std::vector<LabelVox>* out) {
    const rw_pyramid* py = t->pyr;
    const int K = py->K;
    const double scale = std::ldexp(1.0, -(K - k));
    const auto& d = py->dims[k];
    std::unordered_map<int64_t, LabelKey> m;
    std::vector<int64_t> order;
    const size_t n = t->lab_val.size();
    for (size_t i = 0; i < n; ++i) {
        const double fx = std::floor(t->lab_xyz[3 * i] * scale), fy = std::floor(t->lab_xyz[3 * i + 1] * scale),
                     fz = std::floor(t->lab_xyz[3 * i + 2] * scale);
        if (!(fx >= 0 && fy >= 0 && fz >= 0 && fx < d[0] && fy < d[1] && fz < d[2])) continue;
        const int64_t key = ((int64_t)fz * d[1] + (int64_t)fy) * d[0] + (int64_t)fx;
        auto it = m.find(key);
        const int32_t c = t->lab_cls[i];
        if (it == m.end()) {
            m[key] = LabelKey{t->lab_val[i], 0, t->lab_added[i] ? 1 : 0, c};
            order.push_back(key);
        } else {
            if (it->second.value != t->lab_val[i]) it->second.conflict = 1;
            if (c >= 0 && it->second.cls >= 0 && c != it->second.cls) it->second.conflict = 1;
            if (it->second.cls < 0) it->second.cls = c;
            if (t->lab_added[i]) it->second.added = 1;
        }
    }
    out->clear();
    for (int64_t key : order) {
        const LabelKey& L = m[key];
        LabelVox v;
        v.x = (int)(key % d[0]);
        v.y = (int)((key / d[0]) % d[1]);
        v.z = (int)(key / ((int64_t)d[0] * d[1]));
        v.value = L.value;
        v.flags = L.conflict ? (1 | (L.added ? 2 : 0)) : 0;
        out->push_back(v);
    }
}

void children(const rw_tree* t, int k, const std::array<int, 3>& b, std::vector<std::array<int, 3>>* out) {
    const TreeLevel& C = t->L[k + 1];
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                std::array<int, 3> c = {2 * b[0] + dx, 2 * b[1] + dy, 2 * b[2] + dz};
                if (c[0] < C.nbx && c[1] < C.nby && c[2] < C.nbz) out->push_back(c);
            }
}

BrickJob make_job(const rw_tree* t, int k, const std::array<int, 3>& b) {
    const int s = t->pyr->s;
    const int se = (int)std::floor((double)t->opts.expand * s);
    const int mlo = (se - s) / 2, mhi = se - s - mlo;
    const auto& d = t->pyr->dims[k];
    BrickJob J;
    J.bx = b[0];
    J.by = b[1];
    J.bz = b[2];
    int r0[3], r1[3];
    for (int a = 0; a < 3; ++a) {
        const int lo = b[a] * s;
        r0[a] = std::max(lo - mlo, 0);
        r1[a] = std::min(lo + s + mhi, d[a]);
    }
    J.rx0 = r0[0];
    J.ry0 = r0[1];
    J.rz0 = r0[2];
    J.ex = r1[0] - r0[0];
    J.ey = r1[1] - r0[1];
    J.ez = r1[2] - r0[2];
    J.faces = 0;
    if (k > 0) {
        for (int a = 0; a < 3; ++a) {
            if (r0[a] > 0) J.faces |= 1 << (2 * a);
            if (r1[a] < d[a]) J.faces |= 1 << (2 * a + 1);
        }
    }
    J.pad = 0;
    return J;
}

int64_t brick_index(const TreeLevel& L, const std::array<int, 3>& b) {
    return ((int64_t)b[2] * L.nby + b[1]) * L.nbx + b[0];
}

// One tree's share of a level solve: its node list and rasterised labels
// (device copy).
struct Segment {
    rw_tree* t;
    const std::vector<std::array<int, 3>>* nodes;
    const LabelVox* dlab;
    int nlab;
};

// Solve every node of every segment at level k in batched launches: nodes of
// several trees on one pyramid (equal options) share a batch, each tree
// gathering from its own parent and old field and receiving its own results.
// Contract into the level fields and evaluate the node predicates.
rw_status solve_segments(DevWorkspace* w, int k, const std::vector<Segment>& segs, rw_stats* st) {
    if (segs.empty()) return RW_OK;
    const rw_tree* t0 = segs[0].t;
    const rw_pyramid* py = t0->pyr;
    const auto& d = py->dims[k];
    const int s = py->s;
    const int se = std::max(s, (int)std::floor((double)t0->opts.expand * s));
    // the root's neighbourhood is the whole root level (dims <= s)
    const int E = (k == 0) ? std::max(d[0], std::max(d[1], d[2])) : se;
    const int maxb = t0->opts.batch_bricks ? t0->opts.max_batch : 1;
    const rw_opts o = t0->opts;
    std::vector<std::pair<int, int>> ent;  // (segment, node), segments in order
    for (int g = 0; g < (int)segs.size(); ++g)
        for (int i = 0; i < (int)segs[g].nodes->size(); ++i) ent.push_back({g, i});
    for (size_t off = 0; off < ent.size(); off += maxb) {
        const int nb = (int)std::min<size_t>(maxb, ent.size() - off);
        std::vector<BrickJob> jobs(nb);
        std::vector<int> ext(3 * nb);
        for (int i = 0; i < nb; ++i) {
            const auto& e = ent[off + i];
            jobs[i] = make_job(segs[e.first].t, k, (*segs[e.first].nodes)[e.second]);
            ext[3 * i] = jobs[i].ex;
            ext[3 * i + 1] = jobs[i].ey;
            ext[3 * i + 2] = jobs[i].ez;
        }
        // runs of one segment within the batch: {segment, first, end}
        std::vector<std::array<int, 3>> runs;
        for (int i = 0; i < nb; ++i) {
            const int g = ent[off + i].first;
            if (runs.empty() || runs.back()[0] != g) runs.push_back({g, i, i});
            runs.back()[2] = i + 1;
        }
        BrickJob* djobs = nullptr;
        int *dext = nullptr, *dflags = nullptr;
        float *pg = nullptr, *dstats = nullptr;
        uint8_t* pcode = nullptr;
        double* px = nullptr;
        const int64_t pv = (int64_t)E * E * E;
        RCK(ws_get_t(w, S_JOBS, nb * sizeof(BrickJob), &djobs));
        RCK(ws_get_t(w, S_EXT, nb * 3 * sizeof(int), &dext));
        RCK(ws_get_t(w, S_BFLAGS, nb * sizeof(int), &dflags));
        RCK(ws_get_t(w, S_STATS, nb * 3 * sizeof(float), &dstats));
        RCK(ws_get_t(w, S_POOL_G, pv * nb * 4, &pg));
        RCK(ws_get_t(w, S_POOL_CODE, pv * nb, &pcode));
        RCK(ws_get_t(w, S_POOL_X, pv * nb * 8, &px));
        CK(cudaMemcpyAsync(djobs, jobs.data(), nb * sizeof(BrickJob), cudaMemcpyHostToDevice, w->stream));
        CK(cudaMemcpyAsync(dext, ext.data(), nb * 3 * sizeof(int), cudaMemcpyHostToDevice, w->stream));
        CK(cudaMemsetAsync(dflags, 0, nb * sizeof(int), w->stream));
        Boxes bx;
        bx.nbox = nb;
        bx.nx = bx.ny = bx.nz = E;
        bx.ext = dext;
        auto sub = [&](const std::array<int, 3>& r) {
            Boxes b = bx;
            b.nbox = r[2] - r[1];
            b.ext = dext + 3 * r[1];
            return b;
        };
        for (const auto& r : runs) {
            const rw_tree* t = segs[r[0]].t;
            GatherArgs ga;
            ga.bx = sub(r);
            ga.jobs = djobs + r[1];
            ga.gq = (k == py->K) ? py->leaf : nullptr;
            ga.gf = (k == py->K) ? nullptr : py->lv[k];
            ga.lx = d[0];
            ga.ly = d[1];
            ga.lz = d[2];
            ga.parent = k > 0 ? t->L[k - 1].P : nullptr;
            ga.px = k > 0 ? py->dims[k - 1][0] : 1;
            ga.py = k > 0 ? py->dims[k - 1][1] : 1;
            ga.pz = k > 0 ? py->dims[k - 1][2] : 1;
            ga.init = t->update ? t->L[k].P : nullptr;  // warm start: the previous pass's field (in place)
            ga.g_out = pg + r[1] * pv;
            ga.code_out = pcode + r[1] * pv;
            ga.x_out = px + r[1] * pv;
            CK(counted(launch_gather(ga, w->stream)));
            CK(counted(launch_apply_labels(ga.bx, ga.jobs, segs[r[0]].dlab, segs[r[0]].nlab, ga.code_out, ga.x_out,
                                           dflags + r[1], w->stream)));
        }
        SolveProblem P;
        P.bx = bx;
        P.g = pg;
        P.gtype = G_F32;
        P.code = pcode;
        P.value = nullptr;
        P.x0 = nullptr;
        P.rhs = nullptr;
        P.x_hi = px;
        P.init_x = 0;
        SolveResult R;
        RCK(solve_boxes(w, P, o, &R));
        int bad = 0, nos = 0;
        stats_from(R, o, st, &bad, &nos);
        // an incremental pass updates the field in place: statistics first
        // (against the old values), then the bricks that are not similar
        auto contract = [&](const std::array<int, 3>& r, bool write_pass) -> cudaError_t {
            rw_tree* t = segs[r[0]].t;
            ContractArgs ca;
            ca.bx = sub(r);
            ca.jobs = djobs + r[1];
            ca.s = s;
            ca.x = px + r[1] * pv;
            ca.field = t->L[k].P;
            ca.lx = d[0];
            ca.ly = d[1];
            ca.lz = d[2];
            if (write_pass) {
                ca.old = nullptr;
                ca.stats_only = 0;
                ca.stats = nullptr;
                ca.skip = dflags + r[1];
            } else {
                ca.old = t->update ? t->L[k].P : nullptr;
                ca.stats_only = t->update ? 1 : 0;
                ca.stats = dstats + 3 * r[1];
            }
            return launch_contract(ca, w->stream);
        };
        for (const auto& r : runs) CK(counted(contract(r, false)));
        std::vector<float> hst(3 * nb);
        std::vector<int> hfl(nb);
        CK(cudaMemcpyAsync(hst.data(), dstats, nb * 3 * sizeof(float), cudaMemcpyDeviceToHost, w->stream));
        CK(cudaMemcpyAsync(hfl.data(), dflags, nb * sizeof(int), cudaMemcpyDeviceToHost, w->stream));
        CK(cudaStreamSynchronize(w->stream));
        bool any_update = false;
        for (int i = 0; i < nb; ++i) {
            const auto& e = ent[off + i];
            rw_tree* t = segs[e.first].t;
            TreeLevel& L = t->L[k];
            any_update = any_update || t->update;
            const int64_t bi = brick_index(L, (*segs[e.first].nodes)[e.second]);
            const float mn = hst[3 * i], mx = hst[3 * i + 1], md = hst[3 * i + 2];
            int f = RW_NODE_SOLVED | (hfl[i] & (RW_NODE_CFL | RW_NODE_CFL_ADDED));
            if (R.sc[i].nseed == 0) f |= RW_NODE_NO_SEEDS;
            // Sec. IV-D1: hom, dt, prunable = (hom or dt) and not cfl
            const bool hom = (mx - mn) < t->opts.t_hom;
            const bool dt = (mn - 0.5f > t->opts.t_bin) || (0.5f - mx > t->opts.t_bin);
            if (hom) f |= RW_NODE_HOM;
            if (dt) f |= RW_NODE_DT;
            const bool cfl = (f & RW_NODE_CFL) != 0;
            if (((hom && t->opts.prune_hom) || (dt && t->opts.prune_dt)) && !cfl) f |= RW_NODE_PRUNABLE;
            // Sec. IV-E: similar = max |new - old| < t_inc and no conflict with added labels
            if (t->update && md < t->opts.t_inc && !(f & RW_NODE_CFL_ADDED)) f |= RW_NODE_SIMILAR;
            L.flags[bi] = f;
            L.mn[bi] = mn;
            L.mx[bi] = mx;
            L.md[bi] = md;
            hfl[i] = (f & RW_NODE_SIMILAR) ? 1 : 0;  // similar bricks keep their old values
            if (st) {
                st->bricks_solved += 1;
                if (cfl) st->bricks_conflict += 1;
            }
        }
        if (any_update) {
            CK(cudaMemcpyAsync(dflags, hfl.data(), nb * sizeof(int), cudaMemcpyHostToDevice, w->stream));
            for (const auto& r : runs)
                if (segs[r[0]].t->update) CK(counted(contract(r, true)));
        }
    }
    return RW_OK;
}

// Whether a level-(k-1) node read by the trilinear upsample of node b of
// level k (parent voxels h-1 .. h+1 around h = X / 2, clamped) changed in the
// current pass.
bool parent_changed(const rw_tree* t, int k, const std::array<int, 3>& b) {
    const rw_pyramid* py = t->pyr;
    const int s = py->s;
    const TreeLevel& P = t->L[k - 1];
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        const int x0 = b[a] * s, x1 = std::min(x0 + s, py->dims[k][a]) - 1;
        lo[a] = std::max(0, (x0 >> 1) - 1) / s;
        hi[a] = std::min(py->dims[k - 1][a] - 1, (x1 >> 1) + 1) / s;
    }
    for (int z = lo[2]; z <= hi[2]; ++z)
        for (int y = lo[1]; y <= hi[1]; ++y)
            for (int x = lo[0]; x <= hi[0]; ++x)
                if (P.changed[((int64_t)z * P.nby + y) * P.nbx + x]) return true;
    return false;
}

// The work of one tree at one level: the nodes to solve, those reused from
// the previous pass, and the level's rasterised labels.
struct LevelWork {
    std::vector<std::array<int, 3>> nodes, reuse;
    std::vector<LabelVox> labs;
};

void level_begin(rw_tree* t, int k, LevelWork* lw) {
    TreeLevel& L = t->L[k];
    lw->nodes.clear();
    lw->reuse.clear();
    if (k == 0) {
        lw->nodes.push_back({0, 0, 0});
    } else {
        lw->nodes = t->resolve;
        lw->reuse = t->reused;
    }
    std::fill(L.flags.begin(), L.flags.end(), 0);
    std::fill(L.mn.begin(), L.mn.end(), 0.0f);
    std::fill(L.mx.begin(), L.mx.end(), 0.0f);
    std::fill(L.md.begin(), L.md.end(), 0.0f);
    std::fill(L.status.begin(), L.status.end(), 0);
    lw->labs.clear();
    rasterize(t, k, &lw->labs);
}

// After the level's solve: node status, change tracking, the level fill and
// the next level's node lists.
rw_status level_end(rw_tree* t, int k, const LevelWork& lw, rw_stats* st, DevWorkspace* w) {
    const rw_pyramid* py = t->pyr;
    TreeLevel& L = t->L[k];
    const auto& d = py->dims[k];
    const auto& nodes = lw.nodes;
    const auto& reuse = lw.reuse;
    std::vector<std::array<int, 3>> nres, nreu;
    for (const auto& b : nodes) {
        const int64_t bi = brick_index(L, b);
        const int f = L.flags[bi];
        const bool similar = (f & RW_NODE_SIMILAR) != 0;
        if (similar) {
            L.status[bi] = 2;
            if (k < py->K) children(t, k, b, &nreu);
            if (st) st->bricks_reused += 1;
        } else {
            L.status[bi] = 1;
            if (f & RW_NODE_PRUNABLE) {
                if (st) st->bricks_pruned += 1;
            } else if (k < py->K) {
                children(t, k, b, &nres);
            }
        }
    }
    for (const auto& b : reuse) {
        const int64_t bi = brick_index(L, b);
        L.status[bi] = 2;
        L.flags[bi] = RW_NODE_REUSED;
        if (k < py->K) children(t, k, b, &nreu);
        if (st) st->bricks_reused += 1;
    }
    // Values that change in this pass: re-solved nodes that are not similar,
    // and absent nodes, except those filled last pass from a parent footprint
    // that has not changed (their values equal the new upsample).  The fill
    // writes only the absent nodes that change (fill status 0).
    std::vector<uint8_t> fst(L.nb);
    for (int64_t i = 0; i < L.nb; ++i) {
        bool ch;
        if (L.status[i] == 1) {
            ch = true;
        } else if (L.status[i] == 2) {
            ch = false;
        } else if (!t->update || !L.filled[i] || k == 0) {
            ch = true;
        } else {
            const std::array<int, 3> b = {(int)(i % L.nbx), (int)((i / L.nbx) % L.nby), (int)(i / ((int64_t)L.nbx * L.nby))};
            ch = parent_changed(t, k, b);
        }
        L.changed[i] = ch;
        if (ch) L.flags[i] |= RW_NODE_CHANGED;
        fst[i] = (L.status[i] == 0 && ch) ? 0 : 1;
        L.filled[i] = L.status[i] == 0;
    }
    uint8_t* dstatus = nullptr;
    RCK(ws_get_t(w, S_STATUS, L.nb, &dstatus));
    CK(cudaMemcpyAsync(dstatus, fst.data(), L.nb, cudaMemcpyHostToDevice, w->stream));
    FillArgs fa;
    fa.field = L.P;
    fa.lx = d[0];
    fa.ly = d[1];
    fa.lz = d[2];
    fa.parent = k > 0 ? t->L[k - 1].P : nullptr;
    fa.px = k > 0 ? py->dims[k - 1][0] : 1;
    fa.py = k > 0 ? py->dims[k - 1][1] : 1;
    fa.pz = k > 0 ? py->dims[k - 1][2] : 1;
    fa.status = dstatus;
    fa.nbx = L.nbx;
    fa.nby = L.nby;
    fa.nbz = L.nbz;
    fa.s = py->s;
    CK(counted(launch_fill(fa, w->stream)));
    CK(cudaStreamSynchronize(w->stream));
    t->resolve = nres;
    t->reused = nreu;
    std::sort(t->resolve.begin(), t->resolve.end());
    t->resolve.erase(std::unique(t->resolve.begin(), t->resolve.end()), t->resolve.end());
    std::sort(t->reused.begin(), t->reused.end());
    t->reused.erase(std::unique(t->reused.begin(), t->reused.end()), t->reused.end());
    return RW_OK;
}

// Level k of every tree in `trees` (one pyramid, equal options): their
// nodes are solved together, batch by batch.
rw_status process_levels(rw_tree* const* trees, int n, int k, rw_stats* st, DevWorkspace* w) {
    std::vector<LevelWork> lw(n);
    size_t nl = 0;
    for (int i = 0; i < n; ++i) {
        level_begin(trees[i], k, &lw[i]);
        nl += lw[i].labs.size();
        if (st) st->bricks_active += (int64_t)lw[i].nodes.size();
    }
    LabelVox* dlab = nullptr;
    RCK(ws_get_t(w, S_LAB, std::max<size_t>(1, nl) * sizeof(LabelVox), &dlab));
    std::vector<Segment> segs;
    size_t o = 0;
    for (int i = 0; i < n; ++i) {
        const size_t m = lw[i].labs.size();
        if (m)
            CK(cudaMemcpyAsync(dlab + o, lw[i].labs.data(), m * sizeof(LabelVox), cudaMemcpyHostToDevice,
                               w->stream));
        segs.push_back({trees[i], &lw[i].nodes, dlab + o, (int)m});
        o += m;
    }
    RCK(solve_segments(w, k, segs, st));
    for (int i = 0; i < n; ++i) RCK(level_end(trees[i], k, lw[i], st, w));
    return RW_OK;
}

rw_status process_level(rw_tree* t, int k, rw_stats* st, DevWorkspace* w) { return process_levels(&t, 1, k, st, w); }

bool same_solver_opts(const rw_opts& a, const rw_opts& b) {
    return a.beta == b.beta && a.w_min == b.w_min && a.tol == b.tol && a.max_iter == b.max_iter &&
           a.precision == b.precision && a.refine_rounds == b.refine_rounds && a.brick_size == b.brick_size &&
           a.expand == b.expand && a.t_hom == b.t_hom && a.t_bin == b.t_bin && a.t_inc == b.t_inc &&
           a.prune_hom == b.prune_hom && a.prune_dt == b.prune_dt && a.iters_per_graph == b.iters_per_graph &&
           a.tile == b.tile && a.batch_bricks == b.batch_bricks && a.max_batch == b.max_batch && a.weight == b.weight;
}

rw_status copy_labels(rw_tree* t, const rw_labels* lab, int added);
rw_status check_labels(const rw_labels* lab);

// Incremental pass (Sec. IV-E) over n trees on one pyramid with equal
// options; added[i] (nullable) holds tree i's new labels.  Level by level the
// nodes of all trees are solved together.
rw_status update_trees(rw_tree* const* trees, int n, const rw_labels* added, rw_stats* stats, void* stream) {
    g_launches = 0;
    const double t0 = now_ms();
    for (int i = 0; i < n; ++i) {
        rw_tree* t = trees[i];
        if (!t) return fail(RW_ERR_INVALID_ARG, "tree %d is NULL", i);
        if (t->refined != t->pyr->K + 1 || t->open_level >= 0)
            return fail(RW_ERR_INVALID_ARG, "tree %d is not fully refined", i);
        if (t->pyr != trees[0]->pyr) return fail(RW_ERR_INVALID_ARG, "trees on different pyramids");
        if (!same_solver_opts(t->opts, trees[0]->opts)) return fail(RW_ERR_INVALID_ARG, "trees with different options");
        for (int j = 0; j < i; ++j)
            if (trees[j] == t) return fail(RW_ERR_INVALID_ARG, "tree %d given twice", i);
        RCK(check_labels(added ? &added[i] : nullptr));
    }
    if (stats) memset(stats, 0, sizeof(*stats));
    for (int i = 0; i < n; ++i) {
        for (auto& a : trees[i]->lab_added) a = 0;
        RCK(copy_labels(trees[i], added ? &added[i] : nullptr, 1));
    }
    DevWorkspace* w = nullptr;
    RCK(enter(&w, stream));
    for (int i = 0; i < n; ++i) {
        trees[i]->update = 1;
        trees[i]->resolve.clear();
        trees[i]->reused.clear();
        trees[i]->refined = 0;
    }
    for (int k = 0; k <= trees[0]->pyr->K; ++k) {
        RCK(process_levels(trees, n, k, stats, w));
        for (int i = 0; i < n; ++i) trees[i]->refined = k + 1;
    }
    for (int i = 0; i < n; ++i) {
        trees[i]->update = 0;
        for (auto& a : trees[i]->lab_added) a = 0;
    }
    RCK(leave(w));
    if (stats) {
        stats->ms = now_ms() - t0;
        stats->launches = g_launches;
    }
    return RW_OK;
}

rw_status check_labels(const rw_labels* lab) {
    if (!lab || lab->n <= 0) return RW_OK;
    if (!lab->xyz || !lab->value) return fail(RW_ERR_INVALID_ARG, "labels with NULL arrays");
    if (is_device_ptr(lab->xyz) || is_device_ptr(lab->value) || (lab->cls && is_device_ptr(lab->cls)))
        return fail(RW_ERR_INVALID_ARG, "labels must be in host memory");
    return RW_OK;
}

rw_status copy_labels(rw_tree* t, const rw_labels* lab, int added) {
    RCK(check_labels(lab));
    if (!lab || lab->n <= 0) return RW_OK;
    for (int64_t i = 0; i < lab->n; ++i) {
        t->lab_xyz.push_back(lab->xyz[3 * i]);
        t->lab_xyz.push_back(lab->xyz[3 * i + 1]);
        t->lab_xyz.push_back(lab->xyz[3 * i + 2]);
        t->lab_val.push_back(lab->value[i]);
        t->lab_added.push_back((uint8_t)added);
        t->lab_cls.push_back(lab->cls ? lab->cls[i] : -1);
    }
    return RW_OK;
}

// A level refined in parts: start the pass at level 0 (labels stored as by
// rw_refine_level), open the level's node lists.
rw_status open_parts(rw_tree* t, int k, const rw_labels* labels) {
    if (k < 0 || k > t->pyr->K) return fail(RW_ERR_INVALID_ARG, "level %d out of range", k);
    if (t->open_level == k) return RW_OK;
    if (t->open_level >= 0) return fail(RW_ERR_INVALID_ARG, "level %d is open", t->open_level);
    if (k != 0 && k != t->refined) return fail(RW_ERR_INVALID_ARG, "levels must be refined in order");
    if (k == 0) {
        if (labels) {
            t->lab_xyz.clear();
            t->lab_val.clear();
            t->lab_added.clear();
            t->lab_cls.clear();
            RCK(copy_labels(t, labels, 0));
        }
        t->update = 0;
        t->refined = 0;
        t->resolve.clear();
        t->reused.clear();
    }
    LevelWork lw;
    level_begin(t, k, &lw);
    t->open_level = k;
    t->open_nodes = lw.nodes;
    t->open_reuse = lw.reuse;
    t->open_labs = lw.labs;
    t->open_have.assign(lw.nodes.size(), 0);
    return RW_OK;
}

// Positions of `n` brick indices in the open level's node list; `want_have`:
// every node must (1) or must not (0) be present already.
rw_status open_positions(const rw_tree* t, int k, const int64_t* nodes, int64_t n, int want_have,
                         std::vector<int64_t>* pos) {
    if (t->open_level != k) return fail(RW_ERR_INVALID_ARG, "level %d is not open", k);
    if (n < 0 || (n > 0 && !nodes)) return fail(RW_ERR_INVALID_ARG, "bad node list");
    const TreeLevel& L = t->L[k];
    std::unordered_map<int64_t, int64_t> at;
    for (size_t i = 0; i < t->open_nodes.size(); ++i) at[brick_index(L, t->open_nodes[i])] = (int64_t)i;
    pos->resize(n);
    std::vector<uint8_t> seen(t->open_nodes.size(), 0);
    for (int64_t i = 0; i < n; ++i) {
        auto it = at.find(nodes[i]);
        if (it == at.end()) return fail(RW_ERR_INVALID_ARG, "node %lld is not a node of level %d in this pass",
                                        (long long)nodes[i], k);
        if (seen[it->second]) return fail(RW_ERR_INVALID_ARG, "node %lld listed twice", (long long)nodes[i]);
        seen[it->second] = 1;
        if ((int)t->open_have[it->second] != want_have)
            return fail(RW_ERR_INVALID_ARG, want_have ? "node %lld is not present in this tree"
                                                      : "node %lld is already present in this tree",
                        (long long)nodes[i]);
        (*pos)[i] = it->second;
    }
    return RW_OK;
}

}  // namespace

extern "C" {

rw_status rw_build_pyramid(const rw_volume* vol, int32_t brick_size, rw_pyramid** out, void* stream) {
    return rw_build_pyramid_ex(vol, brick_size, 0, out, stream);
}

rw_status rw_build_pyramid_ex(const rw_volume* vol, int32_t brick_size, int32_t flags, rw_pyramid** out,
                              void* stream) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (!out) return fail(RW_ERR_INVALID_ARG, "out is NULL");
    if (flags & ~(RW_PYR_LEAF_HOST | RW_PYR_HOST_ALL))
        return fail(RW_ERR_INVALID_ARG, "unknown pyramid flags 0x%x", flags);
    *out = nullptr;
    int64_t nvox = 0, batch = 1;
    RCK(check_volume(vol, &nvox, &batch));
    if (batch != 1) return fail(RW_ERR_INVALID_ARG, "a pyramid is built from one volume");
    if (brick_size < 2) return fail(RW_ERR_INVALID_ARG, "brick_size < 2");
    DevWorkspace* w = nullptr;
    RCK(enter(&w, stream));
    rw_pyramid* py = new rw_pyramid();
    py->s = brick_size;
    std::vector<std::array<int, 3>> dims;
    std::array<int, 3> dd = {(int)vol->dims[0], (int)vol->dims[1], (int)vol->dims[2]};
    dims.push_back(dd);
    while (std::max(dd[0], std::max(dd[1], dd[2])) > brick_size) {
        for (int a = 0; a < 3; ++a) dd[a] = (dd[a] + 1) / 2;
        dims.push_back(dd);
    }
    std::reverse(dims.begin(), dims.end());
    py->dims = dims;
    py->K = (int)dims.size() - 1;
    py->lv.assign(dims.size(), nullptr);
    auto cleanup = [&](rw_status st) {
        rw_pyramid_free(py);
        return st;
    };
    py->host_all = (flags & RW_PYR_HOST_ALL) ? 1 : 0;
    py->leaf_host = (flags & (RW_PYR_LEAF_HOST | RW_PYR_HOST_ALL)) ? 1 : 0;
    py->lv_host.assign(dims.size(), nullptr);
    void* leaf_dev = nullptr;
    cudaError_t e = level_alloc(py->leaf_host, nvox * 2, &leaf_dev, &py->leaf_host_ptr);
    py->leaf = static_cast<uint16_t*>(leaf_dev);
    if (e != cudaSuccess) return cleanup(fail(RW_ERR_OOM, "pyramid leaf: %s", cudaGetErrorString(e)));
    for (int k = 0; k < py->K; ++k) {
        const int64_t n = (int64_t)dims[k][0] * dims[k][1] * dims[k][2];
        void* lv = nullptr;
        e = level_alloc(py->host_all, n * 4, &lv, &py->lv_host[k]);
        py->lv[k] = static_cast<float*>(lv);
        if (e != cudaSuccess) return cleanup(fail(RW_ERR_OOM, "pyramid level %d: %s", k, cudaGetErrorString(e)));
    }
    // the leaf: device input is quantised in place; host input is copied in
    // z-slabs of at most 256 MB, so no device copy of the whole volume is made
    const size_t esz = vol->dtype == RW_U16 ? 2 : 4;
    if (is_device_ptr(vol->data)) {
        e = launch_quantize(vol->data, vol->dtype, nvox, vol->lo, vol->hi, vol->normalize, RW_STORE_UNORM16, py->leaf,
                            w->stream);
    } else {
        const int64_t plane = (int64_t)dd[0] * dd[1];
        const auto& lf = dims[py->K];
        const int64_t pl = (int64_t)lf[0] * lf[1];
        const int64_t zs = std::max<int64_t>(1, ((int64_t)256 << 20) / (pl * (int64_t)esz));
        (void)plane;
        void* buf = nullptr;
        rw_status st = ws_get(w, S_VOL, (size_t)std::min<int64_t>(zs, lf[2]) * pl * esz, &buf);
        if (st != RW_OK) return cleanup(st);
        for (int64_t z0 = 0; z0 < lf[2] && e == cudaSuccess; z0 += zs) {
            const int64_t nz = std::min<int64_t>(zs, lf[2] - z0);
            e = cudaMemcpyAsync(buf, static_cast<const char*>(vol->data) + z0 * pl * esz, nz * pl * esz,
                                cudaMemcpyHostToDevice, w->stream);
            if (e == cudaSuccess)
                e = launch_quantize(buf, vol->dtype, nz * pl, vol->lo, vol->hi, vol->normalize, RW_STORE_UNORM16,
                                    py->leaf + z0 * pl, w->stream);
        }
    }
    for (int k = py->K - 1; k >= 0 && e == cudaSuccess; --k) {
        const auto& f = dims[k + 1];
        if (k == py->K - 1) e = launch_downsample_u16(py->leaf, f[0], f[1], f[2], py->lv[k], w->stream);
        else e = launch_downsample_f32(py->lv[k + 1], f[0], f[1], f[2], py->lv[k], w->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    if (e != cudaSuccess) return cleanup(fail(RW_ERR_CUDA, "pyramid build: %s", cudaGetErrorString(e)));
    cudaGetDevice(&py->device);
    *out = py;
    return RW_OK;
}

rw_status rw_pyramid_info(const rw_pyramid* py, int32_t* n_levels, int64_t* dims) {
    if (!py) return fail(RW_ERR_INVALID_ARG, "pyramid is NULL");
    if (n_levels) *n_levels = py->K + 1;
    if (dims)
        for (int k = 0; k <= py->K; ++k)
            for (int a = 0; a < 3; ++a) dims[3 * k + a] = py->dims[k][a];
    return RW_OK;
}

rw_status rw_pyramid_read_level(const rw_pyramid* py, int32_t level, float* out, void* stream) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (!py || !out || level < 0 || level > py->K) return fail(RW_ERR_INVALID_ARG, "bad pyramid level");
    DevWorkspace* w = nullptr;
    RCK(enter(&w, stream));
    const auto& d = py->dims[level];
    const int64_t n = (int64_t)d[0] * d[1] * d[2];
    const bool dev = is_device_ptr(out);
    float* dst = out;
    if (!dev) RCK(ws_get_t(w, S_OUT, n * 4, &dst));
    if (level == py->K) CK(counted(launch_leaf_to_f32(py->leaf, n, dst, w->stream)));
    else CK(cudaMemcpyAsync(dst, py->lv[level], n * 4, cudaMemcpyDeviceToDevice, w->stream));
    if (!dev) CK(cudaMemcpyAsync(out, dst, n * 4, cudaMemcpyDeviceToHost, w->stream));
    return leave(w);
}

void rw_pyramid_free(rw_pyramid* py) {
    if (!py) return;
    level_free(py->leaf, py->leaf_host_ptr);
    for (size_t k = 0; k < py->lv.size(); ++k)
        level_free(py->lv[k], k < py->lv_host.size() ? py->lv_host[k] : nullptr);
    delete py;
}

rw_status rw_tree_create(const rw_pyramid* py, const rw_opts* opts_in, rw_tree** out) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (!py || !out) return fail(RW_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    rw_opts o;
    if (opts_in) o = *opts_in;
    else rw_opts_default(&o);
    RCK(check_opts(o));
    if (o.brick_size != py->s) return fail(RW_ERR_INVALID_ARG, "opts.brick_size != pyramid brick size");
    rw_tree* t = new rw_tree();
    t->pyr = py;
    t->opts = o;
    t->L.resize(py->K + 1);
    for (int k = 0; k <= py->K; ++k) {
        TreeLevel& L = t->L[k];
        const auto& d = py->dims[k];
        L.nbx = (d[0] + py->s - 1) / py->s;
        L.nby = (d[1] + py->s - 1) / py->s;
        L.nbz = (d[2] + py->s - 1) / py->s;
        L.nb = (int64_t)L.nbx * L.nby * L.nbz;
        const int64_t n = (int64_t)d[0] * d[1] * d[2];
        const bool all = o.leaf_field == RW_FIELDS_HOST || (o.leaf_field == RW_LEAF_AS_PYRAMID && py->host_all);
        const bool host = all || (k == py->K && (o.leaf_field == RW_LEAF_HOST ||
                                                 (o.leaf_field == RW_LEAF_AS_PYRAMID && py->leaf_host)));
        void* p0 = nullptr;
        cudaError_t e = level_alloc(host, n * 4, &p0, &L.P_host);
        L.P = static_cast<float*>(p0);
        if (e == cudaSuccess) e = cudaMemset(L.P, 0, n * 4);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            rw_tree_free(t);
            return fail(RW_ERR_OOM, "tree level %d: %s", k, cudaGetErrorString(e));
        }
        L.flags.assign(L.nb, 0);
        L.mn.assign(L.nb, 0.0f);
        L.mx.assign(L.nb, 0.0f);
        L.md.assign(L.nb, 0.0f);
        L.status.assign(L.nb, 0);
        L.filled.assign(L.nb, 0);
        L.changed.assign(L.nb, 1);
    }
    *out = t;
    return RW_OK;
}

rw_status rw_refine_level(rw_tree* t, int32_t level, const rw_labels* labels, rw_stats* stats, void* stream) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    g_launches = 0;
    const double t0 = now_ms();
    if (!t) return fail(RW_ERR_INVALID_ARG, "tree is NULL");
    if (level < 0 || level > t->pyr->K) return fail(RW_ERR_INVALID_ARG, "level %d out of range", level);
    if (level != 0 && level != t->refined) return fail(RW_ERR_INVALID_ARG, "levels must be refined in order");
    if (t->open_level >= 0) return fail(RW_ERR_INVALID_ARG, "level %d is open (rw_refine_level_finish)", t->open_level);
    if (stats) memset(stats, 0, sizeof(*stats));
    if (level == 0) {
        if (labels) {
            t->lab_xyz.clear();
            t->lab_val.clear();
            t->lab_added.clear();
            t->lab_cls.clear();
            RCK(copy_labels(t, labels, 0));
        }
        t->update = 0;
        t->refined = 0;
        t->resolve.clear();
        t->reused.clear();
    }
    DevWorkspace* w = nullptr;
    RCK(enter(&w, stream));
    RCK(process_level(t, level, stats, w));
    t->refined = level + 1;
    RCK(leave(w));
    if (stats) {
        stats->ms = now_ms() - t0;
        stats->launches = g_launches;
    }
    return RW_OK;
}

rw_status rw_update_seeds(rw_tree* t, const rw_labels* added, rw_stats* stats, void* stream) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (!t) return fail(RW_ERR_INVALID_ARG, "tree is NULL");
    return update_trees(&t, 1, added, stats, stream);
}

rw_status rw_update_seeds_trees(rw_tree* const* trees, int32_t n_trees, const rw_labels* added, rw_stats* stats,
                                void* stream) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (!trees || n_trees < 1) return fail(RW_ERR_INVALID_ARG, "need at least one tree");
    return update_trees(trees, n_trees, added, stats, stream);
}

rw_status rw_tree_read_level(const rw_tree* t, int32_t level, const int64_t box[6], float* out, void* stream) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (!t || !out || level < 0 || level > t->pyr->K) return fail(RW_ERR_INVALID_ARG, "bad arguments");
    const auto& d = t->pyr->dims[level];
    int64_t bb[6] = {0, 0, 0, d[0], d[1], d[2]};
    if (box)
        for (int i = 0; i < 6; ++i) bb[i] = box[i];
    for (int a = 0; a < 3; ++a)
        if (bb[a] < 0 || bb[a + 3] > d[a] || bb[a] > bb[a + 3]) return fail(RW_ERR_INVALID_ARG, "box outside level");
    DevWorkspace* w = nullptr;
    RCK(enter(&w, stream));
    const int64_t n = (bb[3] - bb[0]) * (bb[4] - bb[1]) * (bb[5] - bb[2]);
    const bool dev = is_device_ptr(out);
    float* dst = out;
    if (!dev) RCK(ws_get_t(w, S_OUT, n * 4, &dst));
    CK(counted(launch_read_box(t->L[level].P, d[0], d[1], d[2], bb, dst, w->stream)));
    if (!dev) CK(cudaMemcpyAsync(out, dst, n * 4, cudaMemcpyDeviceToHost, w->stream));
    return leave(w);
}

rw_status rw_trees_argmax(const rw_tree* const* trees, int32_t n_classes, int32_t level, const int64_t box[6],
                          uint8_t* labels_out, float* prob_out, void* stream) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    static_assert(RW_MAX_CLASSES == 8, "ClassFields holds 8 fields");
    if (!trees || !labels_out || n_classes < 2 || n_classes > RW_MAX_CLASSES)
        return fail(RW_ERR_INVALID_ARG, "need 2..%d trees and an output", RW_MAX_CLASSES);
    ClassFields cf{};
    cf.n = n_classes;
    const rw_pyramid* py = nullptr;
    for (int c = 0; c < n_classes; ++c) {
        if (!trees[c]) return fail(RW_ERR_INVALID_ARG, "tree %d is NULL", c);
        if (c == 0) py = trees[c]->pyr;
        else if (trees[c]->pyr != py) return fail(RW_ERR_INVALID_ARG, "trees on different pyramids");
    }
    if (level < 0 || level > py->K) return fail(RW_ERR_INVALID_ARG, "level %d out of range", level);
    for (int c = 0; c < n_classes; ++c) cf.P[c] = trees[c]->L[level].P;
    const auto& d = py->dims[level];
    int64_t bb[6] = {0, 0, 0, d[0], d[1], d[2]};
    if (box)
        for (int i = 0; i < 6; ++i) bb[i] = box[i];
    for (int a = 0; a < 3; ++a)
        if (bb[a] < 0 || bb[a + 3] > d[a] || bb[a] > bb[a + 3]) return fail(RW_ERR_INVALID_ARG, "box outside level");
    DevWorkspace* w = nullptr;
    RCK(enter(&w, stream));
    // device and page-locked host outputs are written by the kernel; other
    // host outputs go through device staging buffers, a slab of z planes (at
    // most 64 Mi voxels) at a time
    const int64_t plane = (bb[3] - bb[0]) * (bb[4] - bb[1]);
    uint8_t* lab_w = labels_out;  // kernel-writable address of the output (or nullptr)
    float* prob_w = prob_out;
    if (!is_device_ptr(labels_out)) lab_w = static_cast<uint8_t*>(pinned_device_alias(labels_out));
    if (prob_out && !is_device_ptr(prob_out)) prob_w = static_cast<float*>(pinned_device_alias(prob_out));
    const bool lab_dev = lab_w != nullptr, prob_dev = !prob_out || prob_w != nullptr;
    const int64_t nz = bb[5] - bb[2];
    const int64_t slab = (lab_dev && prob_dev) ? std::max<int64_t>(nz, 1)
                                               : std::max<int64_t>(1, ((int64_t)1 << 26) / std::max<int64_t>(plane, 1));
    uint8_t* lab_st = nullptr;
    float* prob_st = nullptr;
    if (!lab_dev) RCK(ws_get_t(w, S_CODE, std::max<int64_t>(1, std::min(slab, nz) * plane), &lab_st));
    if (!prob_dev) RCK(ws_get_t(w, S_OUT, std::max<int64_t>(1, std::min(slab, nz) * plane) * 4, &prob_st));
    for (int64_t z0 = 0; z0 < nz; z0 += slab) {
        const int64_t z1 = std::min(nz, z0 + slab);
        const int64_t sb[6] = {bb[0], bb[1], bb[2] + z0, bb[3], bb[4], bb[2] + z1};
        const int64_t off = z0 * plane, m = (z1 - z0) * plane;
        uint8_t* lab = lab_dev ? lab_w + off : lab_st;
        float* prob = prob_out ? (prob_dev ? prob_w + off : prob_st) : nullptr;
        CK(counted(launch_argmax(cf, d[0], d[1], sb, lab, prob, w->stream)));
        if (!lab_dev) CK(cudaMemcpyAsync(labels_out + off, lab_st, m, cudaMemcpyDeviceToHost, w->stream));
        if (!prob_dev) CK(cudaMemcpyAsync(prob_out + off, prob_st, m * 4, cudaMemcpyDeviceToHost, w->stream));
    }
    return leave(w);
}

rw_status rw_trees_argmax_changed(const rw_tree* const* trees, int32_t n_classes, uint8_t* labels_out,
                                  float* prob_out, void* stream) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (!trees || !labels_out || n_classes < 2 || n_classes > RW_MAX_CLASSES)
        return fail(RW_ERR_INVALID_ARG, "need 2..%d trees and an output", RW_MAX_CLASSES);
    ClassFields cf{};
    cf.n = n_classes;
    const rw_pyramid* py = nullptr;
    for (int c = 0; c < n_classes; ++c) {
        if (!trees[c]) return fail(RW_ERR_INVALID_ARG, "tree %d is NULL", c);
        if (c == 0) py = trees[c]->pyr;
        else if (trees[c]->pyr != py) return fail(RW_ERR_INVALID_ARG, "trees on different pyramids");
        if (trees[c]->refined != py->K + 1) return fail(RW_ERR_INVALID_ARG, "tree %d is not fully refined", c);
        cf.P[c] = trees[c]->L[py->K].P;
    }
    uint8_t* lab = is_device_ptr(labels_out) ? labels_out : static_cast<uint8_t*>(pinned_device_alias(labels_out));
    float* prob = nullptr;
    if (prob_out) {
        prob = is_device_ptr(prob_out) ? prob_out : static_cast<float*>(pinned_device_alias(prob_out));
        if (!prob) return fail(RW_ERR_INVALID_ARG, "prob_out must be device or page-locked host memory");
    }
    if (!lab) return fail(RW_ERR_INVALID_ARG, "labels_out must be device or page-locked host memory");
    const TreeLevel& L0 = trees[0]->L[py->K];
    std::vector<int64_t> nodes;
    for (int64_t i = 0; i < L0.nb; ++i) {
        bool ch = false;
        for (int c = 0; c < n_classes && !ch; ++c) ch = trees[c]->L[py->K].changed[i] != 0;
        if (ch) nodes.push_back(i);
    }
    DevWorkspace* w = nullptr;
    RCK(enter(&w, stream));
    if (!nodes.empty()) {
        int64_t* dn = nullptr;
        RCK(ws_get_t(w, S_NODES, nodes.size() * sizeof(int64_t), &dn));
        CK(cudaMemcpyAsync(dn, nodes.data(), nodes.size() * sizeof(int64_t), cudaMemcpyHostToDevice, w->stream));
        const auto& d = py->dims[py->K];
        CK(counted(launch_argmax_nodes(cf, d[0], d[1], d[2], py->s, L0.nbx, L0.nby, dn, (int64_t)nodes.size(), lab,
                                       prob, w->stream)));
    }
    return leave(w);
}

rw_status rw_tree_node_stats(const rw_tree* t, int32_t level, int64_t* n_nodes, int32_t* flags, float* mn, float* mx,
                             float* maxdiff) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (!t || level < 0 || level > t->pyr->K) return fail(RW_ERR_INVALID_ARG, "bad arguments");
    const TreeLevel& L = t->L[level];
    if (n_nodes) *n_nodes = L.nb;
    if (flags) memcpy(flags, L.flags.data(), L.nb * sizeof(int32_t));
    if (mn) memcpy(mn, L.mn.data(), L.nb * sizeof(float));
    if (mx) memcpy(mx, L.mx.data(), L.nb * sizeof(float));
    if (maxdiff) memcpy(maxdiff, L.md.data(), L.nb * sizeof(float));
    return RW_OK;
}

rw_status rw_tree_level_nodes(const rw_tree* t, int32_t level, int64_t* n_nodes, int64_t* nodes) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (!t || !n_nodes) return fail(RW_ERR_INVALID_ARG, "NULL argument");
    if (level < 0 || level > t->pyr->K) return fail(RW_ERR_INVALID_ARG, "level %d out of range", level);
    std::vector<int64_t> ids;
    if (t->open_level == level) {
        for (const auto& b : t->open_nodes) ids.push_back(brick_index(t->L[level], b));
    } else if (level == 0) {
        if (t->open_level >= 0) return fail(RW_ERR_INVALID_ARG, "level %d is open", t->open_level);
        ids.push_back(0);
    } else {
        if (t->open_level >= 0 || level != t->refined)
            return fail(RW_ERR_INVALID_ARG, "level %d is not the next level of the pass", level);
        for (const auto& b : t->resolve) ids.push_back(brick_index(t->L[level], b));
    }
    std::sort(ids.begin(), ids.end());
    if (nodes) std::copy(ids.begin(), ids.end(), nodes);
    *n_nodes = (int64_t)ids.size();
    return RW_OK;
}

rw_status rw_refine_level_nodes(rw_tree* t, int32_t level, const rw_labels* labels, const int64_t* nodes,
                                int64_t n_nodes, rw_stats* stats, void* stream) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    g_launches = 0;
    const double t0 = now_ms();
    if (!t) return fail(RW_ERR_INVALID_ARG, "tree is NULL");
    if (stats) memset(stats, 0, sizeof(*stats));
    if (labels && level != 0) return fail(RW_ERR_INVALID_ARG, "labels are given at level 0");
    RCK(check_labels(labels));
    RCK(open_parts(t, level, labels));
    std::vector<int64_t> pos;
    RCK(open_positions(t, level, nodes, n_nodes, 0, &pos));
    std::vector<std::array<int, 3>> sub;
    for (int64_t i : pos) sub.push_back(t->open_nodes[i]);
    std::sort(sub.begin(), sub.end());
    if (stats) stats->bricks_active = (int64_t)sub.size();
    if (!sub.empty()) {
        DevWorkspace* w = nullptr;
        RCK(enter(&w, stream));
        LabelVox* dlab = nullptr;
        const size_t nl = t->open_labs.size();
        RCK(ws_get_t(w, S_LAB, std::max<size_t>(1, nl) * sizeof(LabelVox), &dlab));
        if (nl) CK(cudaMemcpyAsync(dlab, t->open_labs.data(), nl * sizeof(LabelVox), cudaMemcpyHostToDevice, w->stream));
        std::vector<Segment> segs = {{t, &sub, dlab, (int)nl}};
        RCK(solve_segments(w, level, segs, stats));
        RCK(leave(w));
    }
    for (int64_t i : pos) t->open_have[i] = 1;
    if (stats) {
        stats->ms = now_ms() - t0;
        stats->launches = g_launches;
    }
    return RW_OK;
}

rw_status rw_tree_export_nodes(const rw_tree* t, int32_t level, const int64_t* nodes, int64_t n_nodes, int32_t* flags,
                               float* node_stats, float* values, void* stream) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (!t) return fail(RW_ERR_INVALID_ARG, "tree is NULL");
    std::vector<int64_t> pos;
    RCK(open_positions(t, level, nodes, n_nodes, 1, &pos));
    const TreeLevel& L = t->L[level];
    for (int64_t i = 0; i < n_nodes; ++i) {
        const int64_t bi = nodes[i];
        if (flags) flags[i] = L.flags[bi];
        if (node_stats) {
            node_stats[3 * i] = L.mn[bi];
            node_stats[3 * i + 1] = L.mx[bi];
            node_stats[3 * i + 2] = L.md[bi];
        }
    }
    if (!values || n_nodes == 0) return RW_OK;
    const int s = t->pyr->s;
    const auto& d = t->pyr->dims[level];
    const int64_t nval = n_nodes * (int64_t)s * s * s;
    DevWorkspace* w = nullptr;
    RCK(enter(&w, stream));
    int64_t* dn = nullptr;
    RCK(ws_get_t(w, S_SHARD_N, n_nodes * sizeof(int64_t), &dn));
    CK(cudaMemcpyAsync(dn, nodes, n_nodes * sizeof(int64_t), cudaMemcpyHostToDevice, w->stream));
    const bool dev = is_device_ptr(values);
    float* dst = values;
    if (!dev) RCK(ws_get_t(w, S_SHARD_V, nval * 4, &dst));
    CK(counted(launch_brick_io(L.P, d[0], d[1], d[2], s, L.nbx, L.nby, dn, n_nodes, dst, 1, w->stream)));
    if (!dev) CK(cudaMemcpyAsync(values, dst, nval * 4, cudaMemcpyDeviceToHost, w->stream));
    return leave(w);
}

rw_status rw_tree_import_nodes(rw_tree* t, int32_t level, const int64_t* nodes, int64_t n_nodes, const int32_t* flags,
                               const float* node_stats, const float* values, void* stream) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (!t) return fail(RW_ERR_INVALID_ARG, "tree is NULL");
    if (n_nodes > 0 && (!flags || !node_stats || !values))
        return fail(RW_ERR_INVALID_ARG, "flags, node statistics and values are required");
    std::vector<int64_t> pos;
    RCK(open_positions(t, level, nodes, n_nodes, 0, &pos));
    for (int64_t i = 0; i < n_nodes; ++i)
        if (!(flags[i] & RW_NODE_SOLVED)) return fail(RW_ERR_INVALID_ARG, "imported node %lld was not solved",
                                                      (long long)nodes[i]);
    if (n_nodes == 0) return RW_OK;
    TreeLevel& L = t->L[level];
    const int s = t->pyr->s;
    const auto& d = t->pyr->dims[level];
    const int64_t nval = n_nodes * (int64_t)s * s * s;
    DevWorkspace* w = nullptr;
    RCK(enter(&w, stream));
    int64_t* dn = nullptr;
    RCK(ws_get_t(w, S_SHARD_N, n_nodes * sizeof(int64_t), &dn));
    CK(cudaMemcpyAsync(dn, nodes, n_nodes * sizeof(int64_t), cudaMemcpyHostToDevice, w->stream));
    const float* src = values;
    if (!is_device_ptr(values)) {
        float* st = nullptr;
        RCK(ws_get_t(w, S_SHARD_V, nval * 4, &st));
        CK(cudaMemcpyAsync(st, values, nval * 4, cudaMemcpyHostToDevice, w->stream));
        src = st;
    }
    CK(counted(launch_brick_io(L.P, d[0], d[1], d[2], s, L.nbx, L.nby, dn, n_nodes, const_cast<float*>(src), 0,
                               w->stream)));
    RCK(leave(w));
    for (int64_t i = 0; i < n_nodes; ++i) {
        const int64_t bi = nodes[i];
        L.flags[bi] = flags[i];
        L.mn[bi] = node_stats[3 * i];
        L.mx[bi] = node_stats[3 * i + 1];
        L.md[bi] = node_stats[3 * i + 2];
        t->open_have[pos[i]] = 1;
    }
    return RW_OK;
}

rw_status rw_refine_level_finish(rw_tree* t, int32_t level, rw_stats* stats, void* stream) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    g_launches = 0;
    const double t0 = now_ms();
    if (!t) return fail(RW_ERR_INVALID_ARG, "tree is NULL");
    if (t->open_level != level) return fail(RW_ERR_INVALID_ARG, "level %d is not open", level);
    for (size_t i = 0; i < t->open_have.size(); ++i)
        if (!t->open_have[i])
            return fail(RW_ERR_INVALID_ARG, "node %lld of level %d is neither solved nor imported",
                        (long long)brick_index(t->L[level], t->open_nodes[i]), level);
    if (stats) memset(stats, 0, sizeof(*stats));
    LevelWork lw;
    lw.nodes = t->open_nodes;
    lw.reuse = t->open_reuse;
    DevWorkspace* w = nullptr;
    RCK(enter(&w, stream));
    RCK(level_end(t, level, lw, stats, w));
    RCK(leave(w));
    t->refined = level + 1;
    t->open_level = -1;
    t->open_nodes.clear();
    t->open_reuse.clear();
    t->open_labs.clear();
    t->open_have.clear();
    if (stats) {
        stats->ms = now_ms() - t0;
        stats->launches = g_launches;
    }
    return RW_OK;
}

void rw_tree_free(rw_tree* t) {
    if (!t) return;
    for (auto& L : t->L) {
        level_free(L.P, L.P_host);
    }
    delete t;
}

}  // extern "C"
