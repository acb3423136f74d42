// Uneven batches: many independent operations (each with its own context,
// i.e. ring degree, level and operation) spread over concurrent lanes and
// captured into one CUDA graph.
//
// The paper spreads per-modulus kernels over a stream pool (Sec. 3.1.6);
// here a whole operation is the unit: ops are assigned to lanes by
// longest-processing-time-first on their modular-product count, each lane
// is a stream forked from the caller's stream with its own workspace slice,
// and the lanes join back before the call returns.  Capturing the batch
// once and replaying the graph removes the per-launch host cost.
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"


namespace catfhe {

size_t ws_bytes(const Context &c, int op, uint32_t level, uint32_t count);
int op_mul_relin(Context &c, const Keys &keys, const uint64_t *a, const uint64_t *b,
                 uint64_t *out, uint32_t level, uint32_t count, bool fused, void *ws,
                 size_t ws_bytes_in, cudaStream_t s, const Gather *gth, bool split);
int op_rotate(Context &c, const Keys &keys, const uint64_t *a, uint64_t g, uint64_t *out,
              uint32_t level, uint32_t count, void *ws, size_t ws_bytes_in, cudaStream_t s,
              const Gather *gth, bool split);
int op_rescale(Context &c, const uint64_t *a, uint64_t *out, uint32_t level, uint32_t count,
               void *ws, size_t ws_bytes_in, cudaStream_t s);
int op_add(Context &c, const uint64_t *a, const uint64_t *b, uint64_t *out, uint32_t level,
           uint32_t count, cudaStream_t s);
int op_sub(Context &c, const uint64_t *a, const uint64_t *b, uint64_t *out, uint32_t level,
           uint32_t count, cudaStream_t s);
int op_mul_int(Context &c, const uint64_t *a, int64_t k, uint64_t *out, uint32_t level,
               uint32_t count, cudaStream_t s);
int op_add_const(Context &c, const uint64_t *a, int64_t k, uint64_t *out, uint32_t level,
                 uint32_t count, cudaStream_t s);
int op_drop_level(Context &c, const uint64_t *a, uint32_t level, uint32_t new_level,
                  uint64_t *out, uint32_t count, cudaStream_t s);
int op_mul_plain(Context &c, const uint64_t *a, const uint64_t *pt, uint64_t *out, uint32_t level,
                 uint32_t count, cudaStream_t s);

namespace {

constexpr int kMaxLanes = 32;

struct LanePool {
    bool ready = false;
    cudaStream_t s[kMaxLanes];
    cudaEvent_t done[kMaxLanes];
    cudaEvent_t start;
};

std::mutex g_pool_mu;
LanePool g_pool[64];

int lane_pool(LanePool **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return CATFHE_ECUDA;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    LanePool &p = g_pool[dev];
    if (!p.ready) {
        for (int i = 0; i < kMaxLanes; i++) {
            if (cudaStreamCreateWithFlags(&p.s[i], cudaStreamNonBlocking) != cudaSuccess)
                return CATFHE_ECUDA;
            if (cudaEventCreateWithFlags(&p.done[i], cudaEventDisableTiming) != cudaSuccess)
                return CATFHE_ECUDA;
        }
        if (cudaEventCreateWithFlags(&p.start, cudaEventDisableTiming) != cudaSuccess)
            return CATFHE_ECUDA;
        p.ready = true;
    }
    *out = &p;
    return CATFHE_OK;
}

bool needs_ws(int op) {
    return op == CATFHE_OP_MUL_RELIN || op == CATFHE_OP_MUL_RELIN_RESCALE ||
           op == CATFHE_OP_ROTATE || op == CATFHE_OP_RESCALE;
}

// A device buffer not 16-byte aligned is refused (kernels use 16-byte words).
static bool misaligned(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) != 0; }

int check_op(const catfhe_op &o) {
    if (!o.ctx || !o.a || !o.out) return CATFHE_EINVAL;
    if (misaligned(o.a) || misaligned(o.out) || (o.b && misaligned(o.b))) return CATFHE_EINVAL;
    const Context &c = o.ctx->c;
    if (o.level < 1 || int(o.level) > c.L) return CATFHE_ELEVEL;
    switch (o.op) {
        case CATFHE_OP_MUL_RELIN:
            if (!o.b || !o.keys || o.keys->owner != o.ctx) return CATFHE_EINVAL;
            return o.keys->k->ksk.count(0) ? CATFHE_OK : CATFHE_ENOKEY;
        case CATFHE_OP_MUL_RELIN_RESCALE:
            if (!o.b || !o.keys || o.keys->owner != o.ctx) return CATFHE_EINVAL;
            if (c.scheme != CATFHE_CKKS) return CATFHE_ESCHEME;
            if (o.level < 2) return CATFHE_ELEVEL;
            return o.keys->k->ksk.count(0) ? CATFHE_OK : CATFHE_ENOKEY;
        case CATFHE_OP_ROTATE: {
            if (!o.keys || o.keys->owner != o.ctx) return CATFHE_EINVAL;
            const uint64_t g = o.arg % (2 * c.n);
            if (!(g & 1)) return CATFHE_EINVAL;
            return o.keys->k->ksk.count(g) ? CATFHE_OK : CATFHE_ENOKEY;
        }
        case CATFHE_OP_RESCALE:
            if (c.scheme == CATFHE_BFV) return CATFHE_ESCHEME;
            return o.level >= 2 ? CATFHE_OK : CATFHE_ELEVEL;
        case CATFHE_OP_ADD:
        case CATFHE_OP_SUB:
            return o.b ? CATFHE_OK : CATFHE_EINVAL;
        case CATFHE_OP_MUL_INT:
            return CATFHE_OK;
        case CATFHE_OP_ADD_CONST:
            return c.scheme == CATFHE_BFV ? CATFHE_ESCHEME : CATFHE_OK;
        case CATFHE_OP_DROP:
            return (o.level_out >= 1 && o.level_out <= o.level && o.a != o.out) ? CATFHE_OK
                                                                            : CATFHE_ELEVEL;
        case CATFHE_OP_MUL_PLAIN:
            return o.b ? CATFHE_OK : CATFHE_EINVAL;
        default:
            return CATFHE_EINVAL;
    }
}

// Modular products of one operation (the same counts as the benchmark's
// roofline): limb-NTTs times (N/2) log N, plus per-coefficient products.
double op_cost(const catfhe_op &o) {
    const Context &c = o.ctx->c;
    const double n = double(c.n), lg = double(c.log_n), l = double(o.level), K = double(c.K);
    if (o.op == CATFHE_OP_MUL_PLAIN && c.scheme == CATFHE_BFV)  // two transforms of 2l limbs
        return o.count * (2 * 2 * l * n / 2 * lg + 2 * l * n);
    if (!needs_ws(o.op)) return o.count * 2 * l * n;
    if (o.op == CATFHE_OP_RESCALE) return o.count * ((2 + 2 * (l - 1)) * n / 2 * lg + 4 * l * n);
    const double M = l + K;
    double ntt = l, prod = 4 * l;
    for (int i = 0; i < int(l); i += c.alpha) {
        const double a = std::min<double>(c.alpha, l - i);
        ntt += M - a;
        prod += a + a * (M - a) + 2 * M;
    }
    ntt += 2 * (K + 1) + 2 * l;
    prod += 2 * ((K + 1) + (K + 1) * l) + 2 * l;
    return o.count * (ntt * n / 2 * lg + prod * n);
}

// A unit of work on one lane: one entry, or several single-ciphertext
// entries of the same kind, context, keys, level (and Galois element) merged
// into one gathered operation.
struct Unit {
    std::vector<uint32_t> entries;
};

struct Plan {
    std::vector<Unit> units;
    std::vector<std::vector<uint32_t>> lane_units;
    std::vector<size_t> lane_ws;  // bytes, 256-aligned
    size_t total = 0;
};

bool mergeable(const catfhe_op &o) {
    return o.count == 1 && o.ctx->c.scheme != CATFHE_BFV &&
           (o.op == CATFHE_OP_MUL_RELIN || o.op == CATFHE_OP_MUL_RELIN_RESCALE ||
            o.op == CATFHE_OP_ROTATE);
}

// Merging: compatible entries are split into ceil(group / lanes) sized
// gathers (at most kGatherMax), so a large group still spreads over every
// lane while each launch sequence covers several ciphertexts.
void make_units(const catfhe_op *ops, uint32_t n, uint32_t lanes, std::vector<Unit> &units) {
    std::map<std::tuple<int, const void *, const void *, uint32_t, uint64_t>, std::vector<uint32_t>>
        groups;
    std::vector<uint32_t> order;  // first entry of each group, in submission order
    for (uint32_t i = 0; i < n; i++) {
        const catfhe_op &o = ops[i];
        if (!mergeable(o)) {
            units.push_back(Unit{{i}});
            continue;
        }
        const uint64_t g = o.op == CATFHE_OP_ROTATE ? o.arg % (2 * o.ctx->c.n) : 0;
        auto &v = groups[std::make_tuple(o.op, (const void *)o.ctx, (const void *)o.keys, o.level, g)];
        if (v.empty()) order.push_back(i);
        v.push_back(i);
    }
    for (uint32_t first : order) {
        const catfhe_op &o = ops[first];
        const uint64_t g = o.op == CATFHE_OP_ROTATE ? o.arg % (2 * o.ctx->c.n) : 0;
        const auto &v = groups[std::make_tuple(o.op, (const void *)o.ctx, (const void *)o.keys, o.level, g)];
        const size_t per = std::min<size_t>(kGatherMax, (v.size() + lanes - 1) / lanes);
        for (size_t k = 0; k < v.size(); k += per) {
            Unit u;
            u.entries.assign(v.begin() + k, v.begin() + std::min(v.size(), k + per));
            units.push_back(std::move(u));
        }
    }
}

int plan_batch(const catfhe_op *ops, uint32_t n, uint32_t lanes, Plan &p) {
    if (!ops || n == 0) return CATFHE_EINVAL;
    lanes = std::max<uint32_t>(1, std::min<uint32_t>(std::min<uint32_t>(lanes, n), kMaxLanes));
    for (uint32_t i = 0; i < n; i++) {
        const int rc = check_op(ops[i]);
        if (rc) return rc;
    }
    p.units.clear();
    make_units(ops, n, lanes, p.units);
    const uint32_t nu = uint32_t(p.units.size());
    std::vector<uint32_t> order(nu);
    std::vector<double> cost(nu, 0.0);
    for (uint32_t u = 0; u < nu; u++) {
        order[u] = u;
        for (uint32_t i : p.units[u].entries) cost[u] += op_cost(ops[i]);
    }
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return cost[x] > cost[y]; });
    const uint32_t nl = std::min(lanes, nu);
    p.lane_units.assign(nl, {});
    p.lane_ws.assign(nl, 0);
    std::vector<double> load(nl, 0.0);
    for (uint32_t u : order) {
        const uint32_t l = uint32_t(std::min_element(load.begin(), load.end()) - load.begin());
        load[l] += cost[u];
        p.lane_units[l].push_back(u);
        const catfhe_op &o = ops[p.units[u].entries[0]];
        const uint32_t items = p.units[u].entries.size() > 1 ? uint32_t(p.units[u].entries.size())
                                                             : o.count;
        const size_t w = needs_ws(o.op) ? ws_bytes(o.ctx->c, o.op, o.level, items) : 0;
        p.lane_ws[l] = std::max(p.lane_ws[l], (w + 255) & ~size_t(255));
    }
    // within a lane, run in submission order
    for (auto &v : p.lane_units)
        std::sort(v.begin(), v.end(), [&](uint32_t x, uint32_t y) {
            return p.units[x].entries[0] < p.units[y].entries[0];
        });
    p.total = 0;
    for (size_t w : p.lane_ws) p.total += w;
    return CATFHE_OK;
}

int run_one(const catfhe_op &o, void *ws, size_t ws_bytes_in, cudaStream_t s) {
    Context &c = o.ctx->c;
    switch (o.op) {
        case CATFHE_OP_MUL_RELIN:
            return op_mul_relin(c, *o.keys->k, o.a, o.b, o.out, o.level, o.count, false, ws, ws_bytes_in, s, nullptr, false);
        case CATFHE_OP_MUL_RELIN_RESCALE:
            return op_mul_relin(c, *o.keys->k, o.a, o.b, o.out, o.level, o.count, true, ws, ws_bytes_in, s, nullptr, false);
        case CATFHE_OP_ROTATE:
            return op_rotate(c, *o.keys->k, o.a, o.arg, o.out, o.level, o.count, ws, ws_bytes_in, s, nullptr, false);
        case CATFHE_OP_RESCALE:
            return op_rescale(c, o.a, o.out, o.level, o.count, ws, ws_bytes_in, s);
        case CATFHE_OP_ADD:
            return op_add(c, o.a, o.b, o.out, o.level, o.count, s);
        case CATFHE_OP_SUB:
            return op_sub(c, o.a, o.b, o.out, o.level, o.count, s);
        case CATFHE_OP_MUL_INT:
            return op_mul_int(c, o.a, int64_t(o.arg), o.out, o.level, o.count, s);
        case CATFHE_OP_ADD_CONST:
            return op_add_const(c, o.a, int64_t(o.arg), o.out, o.level, o.count, s);
        case CATFHE_OP_DROP:
            return op_drop_level(c, o.a, o.level, o.level_out, o.out, o.count, s);
        case CATFHE_OP_MUL_PLAIN:
            return op_mul_plain(c, o.a, o.b, o.out, o.level, o.count, s);
        default:
            return CATFHE_EINVAL;
    }
}

int run_unit(const catfhe_op *ops, const Unit &u, void *ws, size_t ws_bytes_in, cudaStream_t s) {
    const catfhe_op &o = ops[u.entries[0]];
    if (u.entries.size() == 1) return o.count ? run_one(o, ws, ws_bytes_in, s) : CATFHE_OK;
    Gather g;
    g.n = uint32_t(u.entries.size());
    for (uint32_t k = 0; k < g.n; k++) {
        const catfhe_op &e = ops[u.entries[k]];
        g.a[k] = e.a;
        g.b[k] = e.b;
        g.out[k] = e.out;
    }
    Context &c = o.ctx->c;
    switch (o.op) {
        case CATFHE_OP_MUL_RELIN:
        case CATFHE_OP_MUL_RELIN_RESCALE:
            return op_mul_relin(c, *o.keys->k, o.a, o.b, o.out, o.level, g.n,
                                o.op == CATFHE_OP_MUL_RELIN_RESCALE, ws, ws_bytes_in, s, &g, false);
        case CATFHE_OP_ROTATE:
            return op_rotate(c, *o.keys->k, o.a, o.arg, o.out, o.level, g.n, ws, ws_bytes_in, s, &g, false);
        default:
            return CATFHE_EINVAL;
    }
}

int run_plan(const catfhe_op *ops, const Plan &p, char *ws, cudaStream_t s) {
    LanePool *pool;
    int rc = lane_pool(&pool);
    if (rc) return rc;
    const size_t lanes = p.lane_units.size();
    if (cudaEventRecord(pool->start, s) != cudaSuccess) return CATFHE_ECUDA;
    size_t off = 0;
    for (size_t l = 0; l < lanes; l++) {
        cudaStream_t ls = pool->s[l];
        if (cudaStreamWaitEvent(ls, pool->start, 0) != cudaSuccess) return CATFHE_ECUDA;
        for (uint32_t u : p.lane_units[l]) {
            rc = run_unit(ops, p.units[u], ws + off, p.lane_ws[l], ls);
            if (rc) return rc;
        }
        off += p.lane_ws[l];
        if (cudaEventRecord(pool->done[l], ls) != cudaSuccess) return CATFHE_ECUDA;
        if (cudaStreamWaitEvent(s, pool->done[l], 0) != cudaSuccess) return CATFHE_ECUDA;
    }
    return CATFHE_OK;
}

}  // namespace
}  // namespace catfhe

struct catfhe_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t nodes = 0;
};

using namespace catfhe;

extern "C" {

size_t catfhe_batch_workspace_bytes(const catfhe_op *ops, uint32_t n, uint32_t lanes) {
    Plan p;
    if (plan_batch(ops, n, lanes, p) != CATFHE_OK) return 0;
    return p.total + 256;
}

int catfhe_run_batch(const catfhe_op *ops, uint32_t n, uint32_t lanes, void *ws, size_t ws_bytes,
                     void *stream) {
    Plan p;
    int rc = plan_batch(ops, n, lanes, p);
    if (rc) return rc;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 15)) return CATFHE_EINVAL;
    if (ws_bytes < p.total) return CATFHE_EWORKSPACE;
    return run_plan(ops, p, static_cast<char *>(ws), static_cast<cudaStream_t>(stream));
}

int catfhe_batch_capture(const catfhe_op *ops, uint32_t n, uint32_t lanes, void *ws,
                         size_t ws_bytes, catfhe_graph **out) {
    if (!out) return CATFHE_EINVAL;
    Plan p;
    int rc = plan_batch(ops, n, lanes, p);
    if (rc) return rc;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 15)) return CATFHE_EINVAL;
    if (ws_bytes < p.total) return CATFHE_EWORKSPACE;
    // one uncaptured run first: builds every constant table the ops need, so
    // the captured run allocates nothing
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return CATFHE_ECUDA;
    rc = run_plan(ops, p, static_cast<char *>(ws), cs);
    if (!rc && cudaStreamSynchronize(cs) != cudaSuccess) rc = CATFHE_ECUDA;
    catfhe_graph *g = nullptr;
    if (!rc) {
        g = new catfhe_graph();
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            rc = CATFHE_ECUDA;
        } else {
            const int rc2 = run_plan(ops, p, static_cast<char *>(ws), cs);
            const cudaError_t e = cudaStreamEndCapture(cs, &g->graph);
            rc = rc2 ? rc2 : (e == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA);
        }
        if (!rc && cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) rc = CATFHE_ECUDA;
        if (!rc) cudaGraphGetNodes(g->graph, nullptr, &g->nodes);
    }
    cudaStreamDestroy(cs);
    if (rc) {
        if (g) {
            if (g->exec) cudaGraphExecDestroy(g->exec);
            if (g->graph) cudaGraphDestroy(g->graph);
            delete g;
        }
        return rc;
    }
    *out = g;
    return CATFHE_OK;
}

int catfhe_graph_launch(catfhe_graph *g, void *stream) {
    if (!g || !g->exec) return CATFHE_EINVAL;
    return cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? CATFHE_OK
                                                                                   : CATFHE_ECUDA;
}

size_t catfhe_graph_nodes(const catfhe_graph *g) { return g ? g->nodes : 0; }

void catfhe_graph_destroy(catfhe_graph *g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

int catfhe_tune_ntt(catfhe_ctx *ctx, uint32_t limbs, void *stream, int32_t *chosen, float *us) {
    if (!ctx) return CATFHE_EINVAL;
    int ch = 0;
    const int rc = tune_ntt(ctx->c, limbs, static_cast<cudaStream_t>(stream), &ch, us);
    if (chosen) *chosen = ch;
    return rc;
}

int catfhe_ntt_schedule(const catfhe_ctx *ctx, uint32_t limbs, int32_t *index, int32_t *count,
                        int32_t shape[4]) {
    if (!ctx || limbs == 0) return CATFHE_EINVAL;
    const int sched = ctx->c.ntt_sched[ntt_class(limbs)];
    if (index) *index = sched;
    if (count) *count = ntt_schedule_count(ctx->c.log_n);
    if (shape) {
        int s[4];
        ntt_schedule_shape(ctx->c.log_n, sched, s);
        for (int i = 0; i < 4; i++) shape[i] = s[i];
    }
    return CATFHE_OK;
}

int catfhe_set_ntt_schedule(catfhe_ctx *ctx, int32_t index) {
    if (!ctx || index < 0 || index >= ntt_schedule_count(ctx->c.log_n)) return CATFHE_EINVAL;
    for (int k = 0; k < kNttClasses; k++) ctx->c.ntt_sched[k] = index;
    return CATFHE_OK;
}

}  // extern "C"
