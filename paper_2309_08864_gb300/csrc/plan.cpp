// plan.cpp -- chunking, rounds, arena layout and op lists (host only).
#include "plan.hpp"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <limits>

namespace so2dr {

bool fast_star3d_supported(int r, int depth);
bool fast_star3d_row_ok(int64_t nx, int esize);


int64_t elem_size(int dtype) {
    switch (dtype) {
        case SO2DR_F64: return 8;
        case SO2DR_F32: return 4;
        case SO2DR_BF16: return 2;
        case SO2DR_F16: return 2;
        default: return 0;
    }
}

int num_coeffs(int ndim, int radius, int kind) {
    if (kind == SO2DR_STAR) return 1 + 2 * radius * ndim;
    if (kind == SO2DR_BOX) {
        int w = 2 * radius + 1, n = 1;
        for (int a = 0; a < ndim; ++a) n *= w;
        return n;
    }
    if (kind == SO2DR_VARCOEF_STAR) return 0;
    return -1;
}

std::vector<int> launch_depths(int k, int k_on) {
    std::vector<int> v;
    for (int j = 0; j < k / k_on; ++j) v.push_back(k_on);
    if (k % k_on) v.push_back(k % k_on);
    return v;
}

int round_steps(int64_t T, int k_off, int t) {
    int64_t rounds = (T + k_off - 1) / k_off;
    if (t == rounds - 1 && T % k_off != 0) return (int)(T % k_off);
    return k_off;
}

double Plan::cell_updates() const {
    int64_t inner = 1;
    int64_t ext[3] = {n0, ny, nx};
    for (int a = 0; a < 3; ++a) {
        bool used = (a == 0) || (a == 1 && ndim == 3) || (a == 2);
        if (!used) continue;
        int64_t m = ext[a] - 2 * r;
        inner *= std::max<int64_t>(0, m);
    }
    return (double)inner * (double)T;
}

// ------------------------------------------------------------------ tracker

void Tracker::access(int res, int64_t lo, int64_t hi, bool write) {
    if (hi > lo) pend_.push_back({res, lo, hi, write});
}

void Tracker::commit(int64_t op, int stream, int64_t wait_op[kNumStreams]) {
    for (int s = 0; s < kNumStreams; ++s) wait_op[s] = -1;
    // 1) waits: latest conflicting op of every other stream
    for (const Pending& p : pend_) {
        for (const Entry& e : res_[p.res]) {
            if (e.hi <= p.lo || e.lo >= p.hi) continue;
            if (!(e.write || p.write)) continue;
            if (e.stream == stream) continue;
            wait_op[e.stream] = std::max(wait_op[e.stream], e.op);
        }
    }
    // 2) record: a write supersedes everything it overlaps (all of it is
    //    ordered before this op, by the waits above or by stream order)
    for (const Pending& p : pend_) {
        std::vector<Entry>& v = res_[p.res];
        if (p.write) {
            std::vector<Entry> keep;
            keep.reserve(v.size() + 2);
            for (const Entry& e : v) {
                if (e.hi <= p.lo || e.lo >= p.hi) { keep.push_back(e); continue; }
                if (e.lo < p.lo) keep.push_back({e.lo, p.lo, e.op, e.stream, e.write});
                if (e.hi > p.hi) keep.push_back({p.hi, e.hi, e.op, e.stream, e.write});
            }
            keep.push_back({p.lo, p.hi, op, stream, true});
            v.swap(keep);
        } else {
            v.push_back({p.lo, p.hi, op, stream, false});
        }
    }
    pend_.clear();
}

// Buffer ids of the out-of-core forward list.
enum { kBufIn = 0, kBufCoef = 1, kBufX = 2, kBufY = 3, kBufOut0 = 4 };
constexpr int kMaxOut = 2;

// Sizes (planes) of the out-of-core forward buffers for the plan's chunking.
static void forward_caps(const Plan& p, int64_t* cap_in, int64_t* cap_x, int64_t* cap_y,
                         int64_t* cap_out) {
    int64_t pmax = 0;
    for (int i = 0; i < p.d; ++i) pmax = std::max(pmax, p.starts[i + 1] - p.starts[i]);
    // Circular input: one chunk's input span plus the next chunk's new planes,
    // so the host-to-device stream can run one chunk ahead of the kernels.
    // Spans grow with the round's steps, so the full round (k' = k_off)
    // bounds the residual one; the pair (last chunk, first chunk of the next
    // round) is covered by the wrap term.
    int64_t cin = 0;
    const int kk = p.k_off;
    for (int i = 0; i < p.d; ++i) {
        ChunkGeom g = chunk_geom(p, i, kk);
        int64_t next_hi = (i + 1 < p.d) ? chunk_geom(p, i + 1, kk).hi
                                        : (p.rounds > 1 ? p.n0 + chunk_geom(p, 0, kk).hi : g.b);
        cin = std::max(cin, p.lookahead ? std::max(g.b - g.a, next_hi - g.a) : g.b - g.a);
    }
    int L = (int)launch_depths(p.k_off, p.k_on).size();
    *cap_in = std::max<int64_t>(cin, 1);
    *cap_x = (L >= 2) ? pmax + 2 * (int64_t)p.r * std::max(0, p.k_off - p.k_on) : 0;
    *cap_y = (L >= 3) ? pmax + 2 * (int64_t)p.r * std::max(0, p.k_off - 2 * p.k_on) : 0;
    *cap_out = pmax;
}

static size_t forward_arena(const Plan& p, std::vector<Buffer>* out) {
    int64_t cin, cx, cy, co;
    forward_caps(p, &cin, &cx, &cy, &co);
    bool vc = p.kind == SO2DR_VARCOEF_STAR;
    int64_t cbytes = (p.dtype == SO2DR_F64) ? 8 : 4;
    std::vector<Buffer> b(kBufOut0 + kMaxOut);
    int64_t off = 0;
    auto place = [&](int id, int64_t cap, int64_t pb, int nf) {
        b[id].offset = off;
        b[id].cap = cap;
        b[id].plane_bytes = pb;
        b[id].nfields = nf;
        off += align_up(cap * pb);
    };
    place(kBufIn, cin, p.plane_bytes, 1);
    place(kBufCoef, vc ? cin : 0, 6 * p.plane_cells * cbytes, 6);
    place(kBufX, cx, p.plane_bytes, 1);
    place(kBufY, cy, p.plane_bytes, 1);
    for (int s = 0; s < kMaxOut; ++s) place(kBufOut0 + s, s < p.n_out ? co : 0, p.plane_bytes, 1);
    off += kAlign;  // device status word
    if (out) *out = b;
    return (size_t)off;
}

size_t forward_arena_bytes(const Plan& p) { return forward_arena(p, nullptr); }

bool build_forward_ooc(const Plan& p, RunList& rl, size_t budget) {
    return build_forward_ooc_ex(p, rl, budget, ForwardOpts());
}

bool build_forward_ooc_ex(const Plan& p, RunList& rl, size_t budget, const ForwardOpts& opt) {
    rl.ops.clear();
    size_t need = forward_arena(p, &rl.bufs);
    rl.arena_bytes = need;
    if (budget && need > budget) return false;
    const int nbuf = (int)rl.bufs.size();
    const bool vc = p.kind == SO2DR_VARCOEF_STAR;
    auto src_of = [&](int t) { return t < (int)opt.src_array.size() ? opt.src_array[t] : 0; };
    auto dst_of = [&](int t) { return t < (int)opt.dst_array.size() ? opt.dst_array[t] : 0; };
    int nhost = opt.coef_array + 1;
    for (int v : opt.src_array) nhost = std::max(nhost, v + 1);
    for (int v : opt.dst_array) nhost = std::max(nhost, v + 1);
    for (int v : opt.state_array) nhost = std::max(nhost, v + 1);
    // host arrays: the grid's source/destination per round, the face fields
    Emitter em(rl, nbuf + nhost, nbuf);
    const int64_t cin = rl.bufs[kBufIn].cap;
    int64_t g = 0;
    for (int t = 0; t < p.rounds; ++t) {
        int kk = round_steps(p.T, p.k_off, t);
        std::vector<int> depths = launch_depths(kk, p.k_on);
        int64_t V = (int64_t)t * p.n0;
        for (int i = 0; i < p.d; ++i, ++g) {
            ChunkGeom cg = chunk_geom(p, i, kk);
            // (Algorithm 1) transfer the chunk's new planes to the GPU
            if (cg.hi > cg.lo) {
                for (int f = opt.zero_copy ? 1 : 0; f < (vc ? 2 : 1); ++f) {
                    int buf = f ? kBufCoef : kBufIn;
                    Op op = make_op(kOpH2D, kStreamH2D, t, i);
                    op.host_array = f ? opt.coef_array : src_of(t);
                    op.nfields = f ? 6 : 1;
                    op.field_elems = p.n0 * p.plane_cells;
                    op.pub.src_buf = kHost;
                    op.pub.src_lo = cg.lo;
                    op.pub.src_hi = cg.hi;
                    op.pub.src_slot0 = cg.lo;
                    op.pub.dst_buf = buf;
                    op.pub.dst_lo = cg.lo;
                    op.pub.dst_hi = cg.hi;
                    op.pub.dst_slot0 = floor_mod(V + cg.lo, cin);
                    em.tr.access(em.host_res(op.host_array), cg.lo, cg.hi, false);
                    add_buf_access(em.tr, buf, cg.lo, cg.hi, op.pub.dst_slot0, cin, true);
                    em.emit(op);
                }
            }
            // (Sec. II-B, Sec. IV-B) the chunk's planes [a, b) now sit in the
            // circular buffer: the lower 2*r*k' of them were sent with the
            // previous chunk (region sharing), so the k'-step trapezoid runs
            // without waiting on any neighbour.
            int64_t in_lo = cg.a, in_hi = cg.b;
            int src = kBufIn;
            int64_t src_slot0 = floor_mod(V + cg.a, cin);
            int m = 0;
            for (size_t j = 0; j < depths.size(); ++j) {
                int dl = depths[j];
                m += dl;
                bool last = j + 1 == depths.size();
                int64_t h = (int64_t)p.r * (kk - m);
                int64_t out_lo = last ? cg.s : std::max<int64_t>(0, cg.s - h);
                int64_t out_hi = last ? cg.e : std::min<int64_t>(p.n0, cg.e + h);
                int dst = last ? kBufOut0 + (int)(g % p.n_out) : ((j % 2 == 0) ? kBufX : kBufY);
                // consecutive chunks alternate between two compute streams so
                // that one chunk's last launch overlaps the next chunk's first
                Op op = make_op(kOpKernel, (g % 2) ? kStreamCompute2 : kStreamCompute, t, i);
                op.fn = kFnStencil;
                op.pub.depth = dl;
                op.pub.edge_lo = in_lo == 0;
                op.pub.edge_hi = in_hi == p.n0;
                op.pub.src_buf = src;
                op.pub.src_lo = in_lo;
                op.pub.src_hi = in_hi;
                op.pub.src_slot0 = src_slot0;
                op.pub.dst_buf = dst;
                op.pub.dst_lo = out_lo;
                op.pub.dst_hi = out_hi;
                op.pub.dst_slot0 = 0;
                int64_t scap = rl.bufs[src].cap;
                add_buf_access(em.tr, src, in_lo, in_hi, src_slot0, scap, false);
                if (opt.zero_copy && j == 0 && cg.hi > cg.lo) {
                    // the new planes come from the host grid and go into the
                    // circular buffer (for the next chunk's shared region)
                    op.host_src = src_of(t);
                    op.host_lo = cg.lo;
                    op.host_hi = cg.hi;
                    em.tr.access(em.host_res(src_of(t)), cg.lo, cg.hi, false);
                    add_buf_access(em.tr, kBufIn, cg.lo, cg.hi, floor_mod(V + cg.lo, cin), cin, true);
                }
                if (vc) {
                    op.aux_buf = kBufCoef;
                    op.aux_lo = cg.a;
                    op.aux_slot0 = floor_mod(V + cg.a, cin);
                    add_buf_access(em.tr, kBufCoef, cg.a, cg.b, op.aux_slot0, cin, false);
                }
                add_buf_access(em.tr, dst, out_lo, out_hi, 0, rl.bufs[dst].cap, true);
                em.emit(op);
                if (!last && t == 0 && j < opt.state_array.size()) {
                    // an intermediate state of a single-step round: its owned
                    // planes go to their own host array
                    Op d = make_op(kOpD2H, kStreamD2H, t, i);
                    d.host_array = opt.state_array[j];
                    d.pub.src_buf = dst;
                    d.pub.src_lo = d.pub.dst_lo = cg.s;
                    d.pub.src_hi = d.pub.dst_hi = cg.e;
                    d.pub.src_slot0 = cg.s - out_lo;
                    d.pub.dst_buf = kHost;
                    d.pub.dst_slot0 = cg.s;
                    add_buf_access(em.tr, dst, cg.s, cg.e, cg.s - out_lo, rl.bufs[dst].cap, false);
                    em.tr.access(em.host_res(d.host_array), cg.s, cg.e, true);
                    em.emit(d);
                }
                src = dst;
                in_lo = out_lo;
                in_hi = out_hi;
                src_slot0 = 0;
            }
            // (Algorithm 1) transfer the chunk back: its owned interior planes
            int64_t dlo = opt.all_planes ? cg.s : std::max<int64_t>(cg.s, p.r);
            int64_t dhi = opt.all_planes ? cg.e : std::min<int64_t>(cg.e, p.n0 - p.r);
            if (dhi > dlo) {
                Op op = make_op(kOpD2H, kStreamD2H, t, i);
                op.host_array = dst_of(t);
                op.pub.src_buf = src;
                op.pub.src_lo = dlo;
                op.pub.src_hi = dhi;
                op.pub.src_slot0 = dlo - cg.s;
                op.pub.dst_buf = kHost;
                op.pub.dst_lo = dlo;
                op.pub.dst_hi = dhi;
                op.pub.dst_slot0 = dlo;
                add_buf_access(em.tr, src, dlo, dhi, dlo - cg.s, rl.bufs[src].cap, false);
                em.tr.access(em.host_res(op.host_array), dlo, dhi, true);
                em.emit(op);
            }
        }
    }
    return true;
}

void build_forward_in_core(const Plan& p, RunList& rl) {
    rl.ops.clear();
    const bool vc = p.kind == SO2DR_VARCOEF_STAR;
    int64_t cbytes = (p.dtype == SO2DR_F64) ? 8 : 4;
    // buffers: 0 = A, 1 = coefficients, 2 = B
    rl.bufs.assign(3, Buffer());
    int64_t off = 0;
    rl.bufs[0] = {off, p.n0, p.plane_bytes, 1};
    off += align_up(p.n0 * p.plane_bytes);
    rl.bufs[1] = {off, vc ? p.n0 : 0, 6 * p.plane_cells * cbytes, 6};
    off += align_up((vc ? p.n0 : 0) * 6 * p.plane_cells * cbytes);
    rl.bufs[2] = {off, p.n0, p.plane_bytes, 1};
    off += align_up(p.n0 * p.plane_bytes);
    off += kAlign;
    rl.arena_bytes = (size_t)off;
    Emitter em(rl, 3 + 2, 3);
    for (int f = 0; f < (vc ? 2 : 1); ++f) {
        Op op = make_op(kOpH2D, kStreamH2D, 0, 0);
        op.host_array = f;
        op.nfields = f ? 6 : 1;
        op.field_elems = p.n0 * p.plane_cells;
        op.pub.src_lo = 0;
        op.pub.src_hi = p.n0;
        op.pub.src_slot0 = 0;
        op.pub.dst_buf = f ? 1 : 0;
        op.pub.dst_lo = 0;
        op.pub.dst_hi = p.n0;
        op.pub.dst_slot0 = 0;
        em.tr.access(em.host_res(f), 0, p.n0, false);
        em.tr.access(f ? 1 : 0, 0, p.n0, true);
        em.emit(op);
    }
    int cur = 0;
    for (int t = 0; t < p.rounds; ++t) {
        int kk = round_steps(p.T, p.k_off, t);
        for (int dl : launch_depths(kk, p.k_on)) {
            int dst = cur == 0 ? 2 : 0;
            Op op = make_op(kOpKernel, kStreamCompute, t, 0);
            op.fn = kFnStencil;
            op.pub.depth = dl;
            op.pub.edge_lo = op.pub.edge_hi = 1;
            op.pub.src_buf = cur;
            op.pub.src_lo = 0;
            op.pub.src_hi = p.n0;
            op.pub.dst_buf = dst;
            op.pub.dst_lo = 0;
            op.pub.dst_hi = p.n0;
            if (vc) {
                op.aux_buf = 1;
                op.aux_lo = 0;
                op.aux_slot0 = 0;
                em.tr.access(1, 0, p.n0, false);
            }
            em.tr.access(cur, 0, p.n0, false);
            em.tr.access(dst, 0, p.n0, true);
            em.emit(op);
            cur = dst;
        }
    }
    if (p.n0 - 2 * p.r > 0) {
        Op op = make_op(kOpD2H, kStreamD2H, p.rounds > 0 ? p.rounds - 1 : 0, 0);
        op.host_array = 0;
        op.pub.src_buf = cur;
        op.pub.src_lo = p.r;
        op.pub.src_hi = p.n0 - p.r;
        op.pub.src_slot0 = p.r;
        op.pub.dst_buf = kHost;
        op.pub.dst_lo = p.r;
        op.pub.dst_hi = p.n0 - p.r;
        op.pub.dst_slot0 = p.r;
        em.tr.access(cur, p.r, p.n0 - p.r, false);
        em.tr.access(em.host_res(0), p.r, p.n0 - p.r, true);
        em.emit(op);
    }
}

// ----------------------------------------------------- result-reuse code

namespace {

// Buffers: slabs A/B for each of two chunk parities, the per-step ring for
// each parity.
enum { kRrA0 = 0, kRrB0 = 1, kRrA1 = 2, kRrB1 = 3, kRrRs0 = 4, kRrRs1 = 5 };

size_t rr_layout(const Plan& p, std::vector<Buffer>* out) {
    int64_t pmax = 0;
    for (int i = 0; i < p.d; ++i) pmax = std::max(pmax, p.starts[i + 1] - p.starts[i]);
    const int64_t slab = pmax + (int64_t)(p.k_off + 2) * p.r;     // planes a chunk's parallelogram spans
    const int64_t ring = (int64_t)(p.k_off + 1) * 2 * p.r;         // top 2r planes of every step
    std::vector<Buffer> b(6);
    int64_t off = 0;
    for (int id = 0; id < 6; ++id) {
        int64_t cap = id < 4 ? slab : ring;
        b[id] = {off, cap, p.plane_bytes, 1};
        off += align_up(cap * p.plane_bytes);
    }
    off += kAlign;
    if (out) *out = b;
    return (size_t)off;
}

}  // namespace

bool build_result_reuse(const Plan& p0, RunList& rl, size_t budget, int* chunks_out) {
    if (p0.rounds <= 0 || p0.n0 - 2 * p0.r < 1) return false;
    Plan p = p0;
    // chunks: as few as fit the budget (at least the plan's floor)
    int64_t M = p.n0 - 2 * p.r;
    int d = std::max(1, p0.d);
    for (; d <= M; ++d) {
        p.d = d;
        partition_planes(p);
        if (!budget || rr_layout(p, nullptr) <= budget) break;
    }
    if (d > M) return false;
    // region sharing of intermediate results needs every chunk to hold the
    // parallelogram's shift plus the shared planes (the working space for
    // halos may not exceed a chunk, Sec. IV-C)
    for (int i = 0; i < p.d; ++i)
        if (p.starts[i + 1] - p.starts[i] < (int64_t)(p.k_off + 2) * p.r) return false;
    rl.ops.clear();
    rl.arena_bytes = rr_layout(p, &rl.bufs);
    const int nbuf = (int)rl.bufs.size();
    Emitter em(rl, nbuf + 1, nbuf);
    const int r = p.r;
    int64_t g = 0;
    for (int t = 0; t < p.rounds; ++t) {
        const int kk = round_steps(p.T, p.k_off, t);
        for (int i = 0; i < p.d; ++i, ++g) {
            const int q = (int)(g % 2);
            const int bufA = q ? kRrA1 : kRrA0, bufB = q ? kRrB1 : kRrB0;
            const int ring_out = q ? kRrRs1 : kRrRs0, ring_in = q ? kRrRs0 : kRrRs1;
            const bool first = i == 0, last = i == p.d - 1;
            const int64_t s = p.starts[i], e = p.starts[i + 1];
            // slot of plane z in the slabs: z - base (base = lowest plane ever held)
            const int64_t base = std::max<int64_t>(0, s - (int64_t)(kk + 1) * r);
            const int comp = (g % 2) ? kStreamCompute2 : kStreamCompute;
            auto d2d = [&](int src, int64_t slo, int64_t sslot, int dst, int64_t dslot, int64_t n, int step) {
                if (n <= 0) return;
                Op op = make_op(kOpD2D, comp, t, i);
                op.pub.depth = step;
                op.pub.src_buf = src;
                op.pub.src_lo = slo;
                op.pub.src_hi = slo + n;
                op.pub.src_slot0 = sslot;
                op.pub.dst_buf = dst;
                op.pub.dst_lo = slo;
                op.pub.dst_hi = slo + n;
                op.pub.dst_slot0 = dslot;
                em.tr.access(src, sslot, sslot + n, false);
                em.tr.access(dst, dslot, dslot + n, true);
                em.emit(op);
            };
            // step 0: the chunk's own planes from the host
            const int64_t hlo = first ? 0 : s, hhi = last ? p.n0 : e;
            {
                Op op = make_op(kOpH2D, kStreamH2D, t, i);
                op.host_array = 0;
                op.pub.src_lo = op.pub.dst_lo = hlo;
                op.pub.src_hi = op.pub.dst_hi = hhi;
                op.pub.src_slot0 = hlo;
                op.pub.dst_buf = bufA;
                op.pub.dst_slot0 = hlo - base;
                em.tr.access(em.host_res(0), hlo, hhi, false);
                em.tr.access(bufA, hlo - base, hhi - base, true);
                em.emit(op);
            }
            int cur = bufA, oth = bufB;
            // region sharing of step j: write my top 2r planes, read the previous chunk's
            auto share = [&](int buf, int j) {
                const int64_t top = last ? p.n0 : e - (int64_t)j * r;  // my range at step j ends here
                if (!last) d2d(buf, top - 2 * r, top - 2 * r - base, ring_out, (int64_t)j * 2 * r, 2 * r, j);
                if (!first) {
                    const int64_t lo = s - (int64_t)(j + 2) * r;     // planes [s - (j+2)r, s - jr)
                    const int64_t clo = std::max<int64_t>(0, lo);
                    Op op = make_op(kOpD2D, comp, t, i);
                    op.pub.depth = j;
                    op.pub.src_buf = ring_in;
                    op.pub.src_lo = clo;
                    op.pub.src_hi = s - (int64_t)j * r;
                    op.pub.src_slot0 = (int64_t)j * 2 * r + (clo - lo);
                    op.pub.dst_buf = buf;
                    op.pub.dst_lo = clo;
                    op.pub.dst_hi = s - (int64_t)j * r;
                    op.pub.dst_slot0 = clo - base;
                    int64_t n = op.pub.src_hi - op.pub.src_lo;
                    if (n > 0) {
                        em.tr.access(ring_in, op.pub.src_slot0, op.pub.src_slot0 + n, false);
                        em.tr.access(buf, op.pub.dst_slot0, op.pub.dst_slot0 + n, true);
                        em.emit(op);
                    }
                }
            };
            share(cur, 0);
            for (int j = 1; j <= kk; ++j) {
                // step j: input planes [s-(j+1)r, e-(j-1)r) -> output [s-jr, e-jr)
                const int64_t a = first ? 0 : s - (int64_t)(j + 1) * r;
                const int64_t b = last ? p.n0 : e - (int64_t)(j - 1) * r;
                const int64_t olo = first ? 0 : a + r, ohi = last ? p.n0 : b - r;
                Op op = make_op(kOpKernel, comp, t, i);
                op.fn = kFnStencil;
                op.pub.depth = 1;
                op.pub.edge_lo = a == 0;
                op.pub.edge_hi = b == p.n0;
                op.pub.src_buf = cur;
                op.pub.src_lo = a;
                op.pub.src_hi = b;
                op.pub.src_slot0 = a - base;
                op.pub.dst_buf = oth;
                op.pub.dst_lo = olo;
                op.pub.dst_hi = ohi;
                op.pub.dst_slot0 = olo - base;
                em.tr.access(cur, a - base, b - base, false);
                em.tr.access(oth, olo - base, ohi - base, true);
                em.emit(op);
                std::swap(cur, oth);
                if (j < kk) share(cur, j);
            }
            // back to the host: the final parallelogram's interior planes
            const int64_t dlo = first ? r : s - (int64_t)kk * r, dhi = last ? p.n0 - r : e - (int64_t)kk * r;
            if (dhi > dlo) {
                Op op = make_op(kOpD2H, kStreamD2H, t, i);
                op.host_array = 0;
                op.pub.src_buf = cur;
                op.pub.src_lo = op.pub.dst_lo = dlo;
                op.pub.src_hi = op.pub.dst_hi = dhi;
                op.pub.src_slot0 = dlo - base;
                op.pub.dst_slot0 = dlo;
                em.tr.access(cur, dlo - base, dhi - base, false);
                em.tr.access(em.host_res(0), dlo, dhi, true);
                em.emit(op);
            }
        }
    }
    if (chunks_out) *chunks_out = p.d;
    return true;
}

// ------------------------------------------------------------- cost model

namespace {

// Cell updates the kernels compute for one plan (trapezoids included), and
// the useful ones.
void trapezoid_work(const Plan& p, double* computed, double* useful) {
    double c = 0, u = 0;
    for (int t = 0; t < p.rounds; ++t) {
        int kk = round_steps(p.T, p.k_off, t);
        std::vector<int> depths = launch_depths(kk, p.k_on);
        for (int i = 0; i < p.d; ++i) {
            ChunkGeom cg = chunk_geom(p, i, kk);
            int64_t lo = cg.a, hi = cg.b;
            int m = 0;
            for (int dl : depths) {
                for (int l = 1; l <= dl; ++l) {
                    int64_t h = (int64_t)p.r * (kk - (m + l));
                    int64_t zlo = std::max<int64_t>(0, cg.s - h), zhi = std::min<int64_t>(p.n0, cg.e + h);
                    (void)lo;
                    (void)hi;
                    c += (double)(zhi - zlo);
                }
                m += dl;
            }
            u += (double)(cg.e - cg.s) * kk;
        }
    }
    *computed = c;
    *useful = u;
}

// Measured in-core rates (cell updates per second, in-plane halo work
// included) of the kernels on one GB300: the register-streaming 3D star kernel
// by radius and depth, and the generic kernel.
double kernel_rate(const Plan& p, int depth) {
    if (p.kind == SO2DR_BOX && p.ndim == 2 && p.dtype != SO2DR_F64 && p.nx % 4 == 0 && depth <= p.max_kon_auto) {
        // 2D box kernel, in-core cell-steps/s measured on 16384^2 FP32
        // (unmeasured depths interpolated)
        static const double b1[9] = {0, 757e9, 1029e9, 1120e9, 1203e9, 1250e9, 1300e9, 1340e9, 1368e9};
        static const double b2[5] = {0, 557e9, 703e9, 745e9, 786e9};
        static const double b3[4] = {0, 371e9, 375e9, 384e9};
        static const double b4[3] = {0, 248e9, 238e9};
        switch (p.r) {
            case 1: return b1[std::min(depth, 8)];
            case 2: return b2[std::min(depth, 4)];
            case 3: return b3[std::min(depth, 3)];
            default: return b4[std::min(depth, 2)];
        }
    }
    bool fast = p.kind == SO2DR_STAR && p.ndim == 3 && p.dtype != SO2DR_F64 && p.nx % 4 == 0 &&
                depth <= p.max_kon_auto;
    if (!fast) return p.dtype == SO2DR_F64 ? 20e9 : 100e9;
    // (in-core, 1024^3 FP32; radius 3 and 4 at depth 2 run 2 rows per warp
    // and 2R = 6 or 8 unrolled phases, far slower than one level)
    if (p.r == 1) {
        const double r1[5] = {0, 815e9, 1280e9, 1470e9, 1510e9};
        return r1[std::min(depth, 4)];
    }
    if (p.r == 2) return depth >= 2 ? 780e9 : 800e9;
    if (p.r == 3) return depth >= 2 ? 320e9 : 545e9;
    return depth >= 2 ? 112e9 : 429e9;
}

double predict_ms(const Plan& p) {
    double comp, use;
    trapezoid_work(p, &comp, &use);
    const double cells_plane = (double)p.plane_cells;
    const bool vc = p.kind == SO2DR_VARCOEF_STAR;
    const double in_plane_bytes = (double)p.plane_bytes + (vc ? 6.0 * cells_plane * 4 : 0.0);
    const double host_h2d = (double)p.rounds * p.n0 * in_plane_bytes / (p.bw_h2d * 1e9);
    const double host_d2h = (double)p.rounds * p.interior_planes() * p.plane_bytes / (p.bw_d2h * 1e9);
    // fused out-of-core launches run at 67-75% of the in-core rate for chunks
    // of 35-45 planes (each launch fills and drains the pipeline of its fused
    // levels), and at nearly all of it for chunks of thousands of rows;
    // single-step launches keep the in-core rate
    const double pavg = (double)p.interior_planes() / std::max(1, p.d);
    const double eff = p.k_on > 1 ? std::max(0.6, pavg / (pavg + 15.0)) : 1.0;
    const double kernel = comp * cells_plane / (eff * kernel_rate(p, p.k_on));
    const int L = (int)launch_depths(p.k_off, p.k_on).size();
    const double units = (double)std::max(1, p.d * p.rounds);
    const double t_launch = kernel / (units * L), t_d2h_chunk = host_d2h / units;
    // without look-ahead a chunk's transfer waits for the previous chunk's
    // first launch; with one output slab a chunk's last launch waits for the
    // previous chunk's device-to-host copy
    const double h2d_stall = p.lookahead ? 0.0 : units * t_launch;
    const double out_stall = p.n_out >= 2 ? 0.0 : units * std::max(0.0, t_d2h_chunk - t_launch * (L - 1));
    const double hbm = (double)p.rounds * p.n0 * p.plane_bytes * (2.0 + 2.0 * L) / (p.bw_hbm * 1e9);
    const double body = std::max(std::max(host_h2d + h2d_stall, host_d2h), std::max(kernel + out_stall, hbm));
    const double fill = body / units * 2.0;
    return (body + fill) * 1e3;
}

}  // namespace

// ------------------------------------------------------------- build_plan

void partition_planes(Plan& p) {
    int64_t M = p.n0 - 2 * p.r;
    p.starts.assign(p.d + 1, 0);
    for (int i = 1; i < p.d; ++i) p.starts[i] = p.r + (M * i) / p.d;
    p.starts[0] = 0;
    p.starts[p.d] = p.n0;
}

// Smallest d >= dmin whose buffers fit (binary search: the buffers shrink as
// d grows); returns 0 if none.
static int fit_chunks(Plan& p, int dmin) {
    int64_t M = p.n0 - 2 * p.r;
    int dmax = (int)std::max<int64_t>(1, M);
    int lo = std::max(1, dmin);
    if (lo > dmax) return 0;
    auto fits = [&](int d) {
        p.d = d;
        partition_planes(p);
        return !p.budget || forward_arena(p, nullptr) <= p.budget;
    };
    if (!fits(dmax)) return 0;
    if (fits(lo)) return lo;
    int a = lo, b = dmax;  // fits(a) false, fits(b) true
    while (b - a > 1) {
        int m = a + (b - a) / 2;
        if (fits(m)) b = m; else a = m;
    }
    p.d = b;
    partition_planes(p);
    return b;
}

int build_plan(Plan& p, int ndim, const int64_t* dims, int radius, int kind, const double* coeffs,
               int ncoeffs, int64_t T, int min_chunks, int k_on, int k_off, size_t budget,
               int dtype, double bw_h2d, double bw_d2h, double bw_hbm, std::string* err,
               const PlanSearch* search) {
    auto fail = [&](int code, const char* m) { if (err) *err = m; return code; };
    if (ndim != 2 && ndim != 3) return fail(SO2DR_E_INVAL, "ndim must be 2 or 3");
    if (!dims) return fail(SO2DR_E_INVAL, "dims is NULL");
    if (radius < 1 || radius > kMaxRadius) return fail(SO2DR_E_INVAL, "radius must be 1..4");
    if (kind < SO2DR_STAR || kind > SO2DR_VARCOEF_STAR) return fail(SO2DR_E_INVAL, "unknown stencil kind");
    if (elem_size(dtype) == 0) return fail(SO2DR_E_INVAL, "unknown storage dtype");
    if (T < 0) return fail(SO2DR_E_INVAL, "time_steps must be >= 0");
    if (min_chunks < 1) return fail(SO2DR_E_INVAL, "min_chunks must be >= 1");
    if (k_on < 0 || k_on > kMaxKon) return fail(SO2DR_E_INVAL, "k_on must be 0..16");
    if (k_off < 0) return fail(SO2DR_E_INVAL, "k_off must be >= 0");
    if (kind == SO2DR_BOX && ndim != 2) return fail(SO2DR_E_UNSUPPORTED, "box stencils are provided in 2D");
    if (kind == SO2DR_VARCOEF_STAR && (ndim != 3 || radius != 1))
        return fail(SO2DR_E_UNSUPPORTED, "the variable-coefficient stencil is the 3D 7-point star");
    if (kind == SO2DR_VARCOEF_STAR && (dtype == SO2DR_BF16 || dtype == SO2DR_F16))
        return fail(SO2DR_E_UNSUPPORTED, "variable coefficients need F32 or F64 storage");
    if (k_on > p.max_kon)
        return fail(SO2DR_E_UNSUPPORTED, "k_on exceeds the deepest fused kernel for this stencil");
    int nc = num_coeffs(ndim, radius, kind);
    if (kind != SO2DR_VARCOEF_STAR) {
        if (!coeffs || ncoeffs != nc) return fail(SO2DR_E_INVAL, "coefficient count does not match the stencil");
        for (int i = 0; i < nc; ++i)
            if (!std::isfinite(coeffs[i])) return fail(SO2DR_E_INVAL, "non-finite coefficient");
    }
    for (int a = 0; a < ndim; ++a)
        if (dims[a] < 1) return fail(SO2DR_E_INVAL, "dims must be >= 1");
    if (dims[0] > (int64_t)1 << 31) return fail(SO2DR_E_UNSUPPORTED, "axis 0 longer than 2^31");
    p.ndim = ndim;
    p.n0 = dims[0];
    p.ny = ndim == 3 ? dims[1] : 1;
    p.nx = ndim == 3 ? dims[2] : dims[1];
    if (p.nx > (int64_t)1 << 31 || p.ny > (int64_t)1 << 31) return fail(SO2DR_E_UNSUPPORTED, "axis too long");
    p.r = radius;
    p.kind = kind;
    p.dtype = dtype;
    p.coeffs.assign(coeffs ? coeffs : nullptr, coeffs ? coeffs + std::max(0, nc) : nullptr);
    p.T = T;
    p.elem_bytes = elem_size(dtype);
    p.plane_cells = p.ny * p.nx;
    p.plane_bytes = p.plane_cells * p.elem_bytes;
    p.budget = budget;
    if (bw_h2d > 0) p.bw_h2d = bw_h2d;
    if (bw_d2h > 0) p.bw_d2h = bw_d2h;
    if (bw_hbm > 0) p.bw_hbm = bw_hbm;
    if (p.n0 - 2 * p.r < 1) {
        // no interior plane: nothing ever changes; a one-chunk plan with no rounds
        p.k_off = std::max(1, k_off);
        p.k_on = std::max(1, k_on);
        p.rounds = 0;
        p.d = 1;
        partition_planes(p);
    } else if (T == 0) {
        p.k_off = std::max(1, k_off);
        p.k_on = std::max(1, std::min(k_on ? k_on : 1, p.k_off));
        p.rounds = 0;
        p.d = std::min<int64_t>(min_chunks, p.n0 - 2 * p.r);
        partition_planes(p);
    } else {
        std::vector<int> kons, koffs;
        if (k_on) kons.push_back(k_on);
        else
            for (int v : {1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 16})
                if (v <= p.max_kon && v <= p.max_kon_auto) kons.push_back(v);
        if (k_off) koffs.push_back(k_off);
        else {
            for (int64_t v = 1; v <= std::min<int64_t>(T, 64); ++v) koffs.push_back((int)v);
            for (int64_t v : {80, 96, 112, 128, 160, 192, 256, 320, 384, 512, 640, 1024})
                if (v < T) koffs.push_back((int)v);
            if (T > 64) koffs.push_back((int)std::min<int64_t>(T, 1 << 30));
        }
        double best = std::numeric_limits<double>::infinity();
        int bko = 0, bkn = 0, bd = 0, bla = 1, bno = 2;
        std::vector<Candidate> feasible;
        // buffer options (look-ahead, output slabs); SO2DR_LOOKAHEAD / SO2DR_NOUT pin one
        const char* ela = std::getenv("SO2DR_LOOKAHEAD");
        const char* eno = std::getenv("SO2DR_NOUT");
        const int fla = search && search->lookahead >= 0 ? search->lookahead : (ela ? std::atoi(ela) : -1);
        const int fno = search && search->n_out >= 0 ? search->n_out : (eno ? std::atoi(eno) : -1);
        std::vector<std::pair<int, int>> opts;
        for (int la : {1, 0})
            for (int no : {2, 1})
                if ((fla < 0 || fla == la) && (fno < 0 || fno == no)) opts.push_back({la, no});
        if (opts.empty()) opts.push_back({1, 2});
        for (int ko : koffs) {
            for (int kn : kons) {
                if (kn > ko && koffs.size() > 1) continue;
                for (auto [la, no] : opts) {
                    Plan q = p;
                    q.k_off = ko;
                    q.k_on = std::min(kn, ko);
                    q.rounds = (int)((T + ko - 1) / ko);
                    q.lookahead = la;
                    q.n_out = no;
                    int d = fit_chunks(q, min_chunks);
                    if (!d) continue;
                    double ms = predict_ms(q);
                    Candidate c;
                    c.k_off = q.k_off;
                    c.k_on = q.k_on;
                    c.d = d;
                    c.lookahead = la;
                    c.n_out = no;
                    c.predicted_ms = ms;
                    feasible.push_back(c);
                    if (search && search->ranked) search->ranked->push_back(c);
                    if (ms < best) best = ms;
                }
            }
        }
        // Among the candidates predicted within 2% of the best, take the ones
        // with the fewest rounds (least host-link traffic); among those
        // predicted within 1% of their lowest, the smallest k_off (least
        // redundant work, when the link bounds them alike), then the lowest
        // prediction: the model cannot tell them apart, and the host link,
        // shared with the rest of the host, is the most variable resource.
        int brounds = std::numeric_limits<int>::max();
        for (const Candidate& c : feasible)
            if (c.predicted_ms <= 1.02 * best) brounds = std::min(brounds, (int)((T + c.k_off - 1) / c.k_off));
        double bmin = std::numeric_limits<double>::infinity();
        for (const Candidate& c : feasible)
            if (c.predicted_ms <= 1.02 * best && (int)((T + c.k_off - 1) / c.k_off) == brounds)
                bmin = std::min(bmin, c.predicted_ms);
        double bms = std::numeric_limits<double>::infinity();
        for (const Candidate& c : feasible) {
            if (c.predicted_ms > 1.02 * best || (int)((T + c.k_off - 1) / c.k_off) != brounds) continue;
            if (c.predicted_ms > 1.01 * bmin) continue;
            if (!bd || c.k_off < bko || (c.k_off == bko && c.predicted_ms < bms)) {
                bms = c.predicted_ms;
                bko = c.k_off;
                bkn = c.k_on;
                bd = c.d;
                bla = c.lookahead;
                bno = c.n_out;
            }
        }
        if (!bd) return fail(SO2DR_E_INFEASIBLE, "no chunking fits the device budget");
        p.k_off = bko;
        p.k_on = bkn;
        p.lookahead = bla;
        p.n_out = bno;
        p.rounds = (int)((T + bko - 1) / bko);
        p.d = bd;
        partition_planes(p);
    }
    if (!build_forward_ooc(p, p.ooc, p.budget))
        return fail(SO2DR_E_INFEASIBLE, "no chunking fits the device budget");
    if (p.kind == SO2DR_VARCOEF_STAR && p.budget && p.n0 - 2 * p.r >= 1) {
        // the adjoint's single-step rounds must fit as well (at the most chunks)
        Plan q = p;
        q.d = (int)std::max<int64_t>(1, p.n0 - 2 * p.r);
        partition_planes(q);
        if (adjoint_arena_bytes(q) > p.budget)
            return fail(SO2DR_E_INFEASIBLE, "the adjoint rounds do not fit the device budget");
    }
    build_forward_in_core(p, p.ic);
    if (p.kind != SO2DR_VARCOEF_STAR && p.rounds > 0)
        if (!build_result_reuse(p, p.rr, p.budget, &p.rr_chunks)) p.rr_chunks = 0;
    // zero-copy input: the first launch of every chunk must run the 3D star
    // kernel (the one that can read mapped host planes)
    p.zc_ok = false;
    if (p.kind == SO2DR_STAR && p.ndim == 3 && p.dtype != SO2DR_F64 && p.rounds > 0 &&
        fast_star3d_row_ok(p.nx, (int)p.elem_bytes) && !std::getenv("SO2DR_GENERIC_KERNEL")) {
        bool all_fast = true;
        for (int t = 0; t < p.rounds; ++t) {
            const int kk = round_steps(p.T, p.k_off, t);
            all_fast = all_fast && fast_star3d_supported(p.r, std::min(kk, p.k_on));
        }
        ForwardOpts zo;
        zo.zero_copy = true;
        p.zc_ok = all_fast && build_forward_ooc_ex(p, p.zc, p.budget, zo);
    }
    int64_t cin, cx, cy, co;
    forward_caps(p, &cin, &cx, &cy, &co);
    p.ring_planes = cin;
    double comp = 0, use = 0;
    if (p.rounds > 0) trapezoid_work(p, &comp, &use);
    p.redundancy = use > 0 ? comp / use - 1.0 : 0.0;
    return SO2DR_OK;
}

}  // namespace so2dr
