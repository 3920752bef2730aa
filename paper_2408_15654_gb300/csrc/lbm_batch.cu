// Many independent lattices advanced together: one launch of the many-lattice kernel per step
// and per group of lattices that share a storage mode, boundary kind and EOS.  The workspace
// holds a descriptor per lattice (TMA maps, constants, buffers, step count) and the tile list
// of each group; the order of the tiles is the schedule.  Runs of graph_steps steps are
// captured once into a CUDA graph and replayed.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "lbm_internal.h"

using namespace lbm_host;

namespace {

struct Group {
    int st;
    bool walls, lang, flow, var_rho;
    int64_t off, count;  // tiles [off, off + count) of the tile list
};

int64_t tiles_of(const lbm_handle* h) { return (int64_t)h->tiles_x * h->tiles_y; }

// Kernel variant of a lattice (the EOS is unused with a prescribed velocity).
Group group_of(const lbm_handle* h) {
    const bool flow = h->prm.velocity == LBM_VELOCITY_SOLVED;
    return Group{h->prm.storage, h->prm.bc_y == LBM_BC_WALLS, flow && h->prm.eos == LBM_EOS_LANGMUIR, flow,
                 flow && h->phys.var_rho != 0, 0, 0};
}

bool same_group(const Group& a, const Group& b) {
    return a.st == b.st && a.walls == b.walls && a.lang == b.lang && a.flow == b.flow && a.var_rho == b.var_rho;
}

// Tile rows of one lattice in launch order: the two edge rows (which patch their boxes and run
// longest) first, then the interior rows.
std::vector<int> row_order(int ntr) {
    std::vector<int> r;
    r.push_back(0);
    if (ntr > 1) r.push_back(ntr - 1);
    for (int k = 1; k + 1 < ntr; ++k) r.push_back(k);
    return r;
}

}  // namespace

struct lbm_batch {
    cudaStream_t stream;
    int max_members;
    int64_t max_tiles;
    lbm::InstDesc* d_desc;
    uint2* d_tiles;
    std::vector<lbm_handle*> members;
    std::vector<Group> groups;
    std::vector<lbm::InstDesc> h_desc;
    cudaEvent_t upload_done;  // the last descriptor upload has read h_desc
    int schedule;
    int graph_steps;
    cudaGraphExec_t graph;
    int64_t launches;
    // warp-specialised kernel: two tile counters in the workspace, used alternately by successive
    // launches (each zeroes the other); the parity of the next launch; that parity after a replay
    // of the graph (which starts by zeroing both)
    int kernel;            // LBM_KERNEL_AUTO, LBM_KERNEL_TILE or LBM_KERNEL_PIPELINED
    int ws_blocks[5];      // resident warp-specialised CTAs per SM of each members' storage mode (0: none)
    int sms;
    unsigned* d_ctr;
    int ctr_parity;
    int graph_end_parity;
};

namespace {

void drop_graph(lbm_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

// Tile list of every group in the order of schedule b->schedule, uploaded to the workspace.
int build_tiles(lbm_batch* b) {
    const int n = (int)b->members.size();
    std::vector<int> order(n);
    for (int k = 0; k < n; ++k) order[k] = k;
    if (b->schedule != LBM_SCHED_MEMBER_ORDER)
        std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
            return tiles_of(b->members[a]) > tiles_of(b->members[c]);
        });
    // group keys in a fixed order
    std::vector<Group> groups;
    for (int k : order) {
        const Group gk = group_of(b->members[k]);
        bool found = false;
        for (const Group& g : groups) found = found || same_group(g, gk);
        if (!found) groups.push_back(gk);
    }
    std::sort(groups.begin(), groups.end(), [](const Group& a, const Group& c) {
        if (a.st != c.st) return a.st < c.st;
        if (a.flow != c.flow) return a.flow < c.flow;
        if (a.var_rho != c.var_rho) return a.var_rho < c.var_rho;
        return a.walls != c.walls ? a.walls < c.walls : a.lang < c.lang;
    });
    std::vector<uint2> tiles;
    for (Group& g : groups) {
        g.off = (int64_t)tiles.size();
        std::vector<int> mem;
        for (int k : order)
            if (same_group(group_of(b->members[k]), g)) mem.push_back(k);
        auto push_row = [&](int k, int ty) {
            const lbm_handle* h = b->members[k];
            for (int tx = 0; tx < h->tiles_x; ++tx) tiles.push_back(make_uint2((unsigned)k, (unsigned)tx | ((unsigned)ty << 16)));
        };
        if (b->schedule == LBM_SCHED_MEMBER_ORDER || b->schedule == LBM_SCHED_LARGEST_FIRST) {
            for (int k : mem)
                for (int ty : row_order(b->members[k]->tiles_y)) push_row(k, ty);
        } else if (b->schedule == LBM_SCHED_EDGES_FIRST) {
            for (int k : mem) {
                const int ntr = b->members[k]->tiles_y;
                push_row(k, 0);
                if (ntr > 1) push_row(k, ntr - 1);
            }
            for (int k : mem)
                for (int ty = 1; ty + 1 < b->members[k]->tiles_y; ++ty) push_row(k, ty);
        } else {  // LBM_SCHED_ROW_INTERLEAVED: row r of every lattice, then row r + 1
            std::vector<std::vector<int>> rows;
            size_t depth = 0;
            for (int k : mem) {
                rows.push_back(row_order(b->members[k]->tiles_y));
                depth = std::max(depth, rows.back().size());
            }
            for (size_t r = 0; r < depth; ++r)
                for (size_t j = 0; j < mem.size(); ++j)
                    if (r < rows[j].size()) push_row(mem[j], rows[j][r]);
        }
        g.count = (int64_t)tiles.size() - g.off;
    }
    if ((int64_t)tiles.size() > b->max_tiles) return fail(LBM_EINVAL, "the members have more tiles than max_tiles");
    if (!tiles.empty())
        LBM_CUDA(cudaMemcpyAsync(b->d_tiles, tiles.data(), tiles.size() * sizeof(uint2), cudaMemcpyHostToDevice,
                                 b->stream));
    LBM_CUDA(cudaStreamSynchronize(b->stream));  // the host tile vector goes out of scope
    b->groups = groups;
    drop_graph(b);
    return LBM_OK;
}

// Descriptors from the members' current host-side state.
int upload_descs(lbm_batch* b) {
    LBM_CUDA(cudaEventSynchronize(b->upload_done));
    const int n = (int)b->members.size();
    for (int k = 0; k < n; ++k) {
        const lbm_handle* h = b->members[k];
        lbm::InstDesc& d = b->h_desc[k];
        std::memset(static_cast<void*>(&d), 0, sizeof(d));
        for (int j = 0; j < 2; ++j) {
            d.tm_fg[j] = h->tm_fg[j];
            d.tm_h[j] = h->tm_h[j];
            d.tm_hist[j] = h->tm_hist[j];
            d.pops[j] = h->pops[j];
            d.hist[j] = h->hist[j];
            d.shist[j] = h->shist[j];
        }
        d.p = h->phys;
        d.status = h->status;
        d.steps = h->steps;
        d.cur = h->cur;
        d.first = h->first;
    }
    if (n)
        LBM_CUDA(cudaMemcpyAsync(b->d_desc, b->h_desc.data(), n * sizeof(lbm::InstDesc), cudaMemcpyHostToDevice,
                                 b->stream));
    LBM_CUDA(cudaEventRecord(b->upload_done, b->stream));
    return LBM_OK;
}

// Kernel of a group: the warp-specialised one unless TILE is chosen or it does not fit.  It hides
// the dependent loads that start every tile; 64-lattice mix on GB300, GLUPS warp-specialised /
// one CTA per tile: FP32 26.3 / 24.5, FP16 31.8 / 31.3, BF16 33.1 / 31.4, FP16_FG 31.4 / 30.0.
bool group_ws(const lbm_batch* b, const Group& g) {
    if (b->ws_blocks[g.st] <= 0 || b->kernel == LBM_KERNEL_TILE) return false;
    return true;
}

// Launch s of a sequence: every group once.
int launch_one(lbm_batch* b, int s) {
    for (const Group& g : b->groups) {
        const bool ws = group_ws(b, g);
        lbm::BatchArgs a;
        a.descs = b->d_desc;
        a.tiles = b->d_tiles + g.off;
        a.s = s;
        a.ntiles = (int)g.count;
        a.ndescs = (int)b->members.size();
        a.ws_ctas = ws ? (int)std::min<int64_t>(g.count, (int64_t)b->ws_blocks[g.st] * b->sms) : 0;
        a.ctr = b->d_ctr + b->ctr_parity;
        a.ctr_next = b->d_ctr + (b->ctr_parity ^ 1);
        cudaError_t e = lbm::launch_batch(g.st, a, lbm::Variant{g.walls, g.lang, g.flow, g.var_rho}, (unsigned)g.count, b->stream);
        if (e != cudaSuccess) return fail(LBM_ECUDA, "batch step launch: %s", cudaGetErrorString(e));
        if (ws) b->ctr_parity ^= 1;
        b->launches++;
    }
    return LBM_OK;
}

int launch_advance(lbm_batch* b, int n) {
    const int count = (int)b->members.size();
    lbm::batch_advance_kernel<<<(count + 127) / 128, 128, 0, b->stream>>>(b->d_desc, count, n);
    LBM_CUDA(cudaGetLastError());
    b->launches++;
    return LBM_OK;
}

int build_graph(lbm_batch* b) {
    drop_graph(b);
    LBM_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    const int64_t before = b->launches;
    const int parity = b->ctr_parity;
    b->ctr_parity = 0;  // every replay starts with both counters zero and the first one in use
    int rc = LBM_OK;
    if (cudaMemsetAsync(b->d_ctr, 0, 2 * sizeof(unsigned), b->stream) != cudaSuccess)
        rc = fail(LBM_ECUDA, "graph capture: counter reset");
    for (int s = 0; s < b->graph_steps && !rc; ++s) rc = launch_one(b, s);
    if (!rc) rc = launch_advance(b, b->graph_steps);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    b->launches = before;  // captured, not launched
    b->graph_end_parity = b->ctr_parity;
    b->ctr_parity = parity;
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(LBM_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return fail(LBM_ECUDA, "graph instantiation: %s", cudaGetErrorString(e));
    }
    return LBM_OK;
}

int check_member(const lbm_batch* b, const lbm_handle* h) {
    if (!h) return fail(LBM_EINVAL, "member is NULL");
    if (h->stream != b->stream) return fail(LBM_EINVAL, "a member was created on another stream than the batch");
    if (h->tiles_x > 0xFFFF || h->tiles_y > 0xFFFF)
        return fail(LBM_EINVAL, "lattice %d x %d has too many tiles along an axis for the batched kernel", h->prm.nx,
                    h->prm.ny);
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_tiles(lbm_handle* const* members, int n, int64_t* tiles) {
    g_err.clear();
    if (n < 0 || (n > 0 && !members) || !tiles) return fail(LBM_EINVAL, "bad arguments");
    int64_t t = 0;
    for (int k = 0; k < n; ++k) {
        if (!members[k]) return fail(LBM_EINVAL, "member %d is NULL", k);
        t += tiles_of(members[k]);
    }
    *tiles = t;
    return LBM_OK;
}

int lbm_batch_workspace_bytes(int max_members, int64_t max_tiles, size_t* bytes) {
    g_err.clear();
    if (max_members < 1 || max_tiles < 1 || !bytes) return fail(LBM_EINVAL, "need max_members >= 1, max_tiles >= 1");
    if (max_members > (1 << 20) || max_tiles > ((int64_t)1 << 32)) return fail(LBM_EINVAL, "batch too large");
    *bytes = align_up((size_t)max_members * sizeof(lbm::InstDesc)) + align_up((size_t)max_tiles * sizeof(uint2)) +
             align_up(2 * sizeof(unsigned));
    return LBM_OK;
}

int lbm_batch_create(int max_members, int64_t max_tiles, void* d_workspace, size_t bytes, void* cuda_stream,
                     lbm_batch** out) {
    g_err.clear();
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    size_t need = 0;
    int rc = lbm_batch_workspace_bytes(max_members, max_tiles, &need);
    if (rc) return rc;
    if (!d_workspace) return fail(LBM_EINVAL, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(d_workspace) % kAlign) return fail(LBM_EINVAL, "workspace not 256-byte aligned");
    if (bytes < need) return fail(LBM_ENOMEM, "workspace of %zu bytes < %zu needed", bytes, need);
    lbm_batch* b = new (std::nothrow) lbm_batch;
    if (!b) return fail(LBM_ENOMEM, "host allocation failed");
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->max_members = max_members;
    b->max_tiles = max_tiles;
    char* ws = static_cast<char*>(d_workspace);
    b->d_desc = reinterpret_cast<lbm::InstDesc*>(ws);
    b->d_tiles = reinterpret_cast<uint2*>(ws + align_up((size_t)max_members * sizeof(lbm::InstDesc)));
    b->d_ctr = reinterpret_cast<unsigned*>(ws + align_up((size_t)max_members * sizeof(lbm::InstDesc)) +
                                           align_up((size_t)max_tiles * sizeof(uint2)));
    b->kernel = LBM_KERNEL_AUTO;
    for (int& w : b->ws_blocks) w = 0;
    b->sms = 0;
    b->ctr_parity = 0;
    b->graph_end_parity = 0;
    b->schedule = LBM_SCHED_LARGEST_FIRST;
    b->graph_steps = 0;
    b->graph = nullptr;
    b->launches = 0;
    b->upload_done = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&b->upload_done, cudaEventDisableTiming);
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_ctr, 0, 2 * sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->upload_done, b->stream);
    if (e != cudaSuccess) {
        if (b->upload_done) cudaEventDestroy(b->upload_done);
        delete b;
        return fail(LBM_ECUDA, "event: %s", cudaGetErrorString(e));
    }
    b->h_desc.resize((size_t)max_members);
    *out = b;
    return LBM_OK;
}

int lbm_batch_set_members(lbm_batch* b, lbm_handle* const* members, int n) {
    g_err.clear();
    if (!b) return fail(LBM_EINVAL, "batch is NULL");
    if (n < 0 || n > b->max_members || (n > 0 && !members)) return fail(LBM_EINVAL, "need 0 <= n <= max_members");
    for (int k = 0; k < n; ++k) {
        int rc = check_member(b, members[k]);
        if (rc) return rc;
        for (int j = 0; j < k; ++j)
            if (members[j] == members[k]) return fail(LBM_EINVAL, "member %d appears twice", k);
    }
    int64_t t = 0;
    lbm_batch_tiles(members, n, &t);
    if (t > b->max_tiles) return fail(LBM_EINVAL, "the members have %lld tiles > max_tiles", (long long)t);
    int ws[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < n; ++k) {
        const int st = members[k]->prm.storage;
        if (ws[st] > 0) continue;
        cudaError_t e = lbm::prepare_batch(st, &ws[st]);
        if (e != cudaSuccess) return fail(LBM_ECUDA, "kernel setup: %s", cudaGetErrorString(e));
    }
    for (int st = 0; st < 5; ++st) b->ws_blocks[st] = ws[st];
    b->members.assign(members, members + n);
    return build_tiles(b);
}

int lbm_batch_set_schedule(lbm_batch* b, int schedule, int graph_steps) {
    g_err.clear();
    if (!b) return fail(LBM_EINVAL, "batch is NULL");
    if (schedule < LBM_SCHED_MEMBER_ORDER || schedule > LBM_SCHED_ROW_INTERLEAVED) return fail(LBM_EINVAL, "bad schedule");
    if (graph_steps < 0 || graph_steps > 4096) return fail(LBM_EINVAL, "graph_steps outside [0, 4096]");
    b->schedule = schedule;
    b->graph_steps = b->stream ? graph_steps : 0;  // the legacy default stream cannot be captured
    return build_tiles(b);
}

int lbm_batch_step(lbm_batch* b, int64_t n) {
    g_err.clear();
    if (!b) return fail(LBM_EINVAL, "batch is NULL");
    if (n < 0) return fail(LBM_EINVAL, "negative step count");
    if (n == 0 || b->members.empty()) return LBM_OK;
    for (const lbm_handle* h : b->members)
        if (!h->initialized) return fail(LBM_ESTATE, "a member has no state (lbm_init_fields first)");
    int rc = upload_descs(b);
    if (rc) return rc;
    int64_t done = 0;
    if (b->graph_steps > 0 && n >= b->graph_steps) {
        if (!b->graph) {
            rc = build_graph(b);
            if (rc) return rc;
        }
        const int K = b->graph_steps;
        for (; n - done >= K; done += K) {
            LBM_CUDA(cudaGraphLaunch(b->graph, b->stream));
            b->launches += (int64_t)K * (int64_t)b->groups.size() + 1;
            b->ctr_parity = b->graph_end_parity;
        }
    }
    const int rem = (int)(n - done);
    for (int s = 0; s < rem && !rc; ++s) rc = launch_one(b, s);
    if (!rc && rem > 0) rc = launch_advance(b, rem);
    if (rc) return rc;
    for (lbm_handle* h : b->members) {
        h->steps += n;
        h->cur = (int)((h->cur + n) & 1);
        h->first = 0;
    }
    return LBM_OK;
}

int lbm_batch_autotune(lbm_batch* b, int trial_steps, int* schedule, int* graph_steps) {
    g_err.clear();
    if (!b) return fail(LBM_EINVAL, "batch is NULL");
    if (trial_steps < 1) return fail(LBM_EINVAL, "trial_steps must be >= 1");
    const int K = b->stream ? 16 : 0;
    struct Cand { int sched, k; float ms; };
    std::vector<Cand> cands;
    for (int s = LBM_SCHED_MEMBER_ORDER; s <= LBM_SCHED_ROW_INTERLEAVED; ++s) cands.push_back(Cand{s, K, 0.f});
    if (K) cands.push_back(Cand{-1, 0, 0.f});  // the best schedule without a graph
    cudaEvent_t e0, e1;
    LBM_CUDA(cudaEventCreate(&e0));
    LBM_CUDA(cudaEventCreate(&e1));
    int rc = LBM_OK;
    int best = -1;
    for (size_t c = 0; c < cands.size() && !rc; ++c) {
        if (cands[c].sched < 0) cands[c].sched = cands[best].sched;
        rc = lbm_batch_set_schedule(b, cands[c].sched, cands[c].k);
        const int trial = cands[c].k ? (trial_steps + cands[c].k - 1) / cands[c].k * cands[c].k : trial_steps;
        if (!rc) rc = lbm_batch_step(b, cands[c].k ? cands[c].k : 1);  // warm-up (builds the graph)
        if (!rc && cudaEventRecord(e0, b->stream) != cudaSuccess) rc = fail(LBM_ECUDA, "event record");
        if (!rc) rc = lbm_batch_step(b, trial);
        if (!rc && cudaEventRecord(e1, b->stream) != cudaSuccess) rc = fail(LBM_ECUDA, "event record");
        if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = fail(LBM_ECUDA, "event synchronize");
        float ms = 0.f;
        if (!rc && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = fail(LBM_ECUDA, "event time");
        cands[c].ms = ms / (float)trial;
        if (!rc && (best < 0 || cands[c].ms < cands[best].ms)) best = (int)c;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    rc = lbm_batch_set_schedule(b, cands[best].sched, cands[best].k);
    if (rc) return rc;
    if (schedule) *schedule = cands[best].sched;
    if (graph_steps) *graph_steps = cands[best].k;
    return LBM_OK;
}

int lbm_batch_set_kernel(lbm_batch* b, int variant) {
    g_err.clear();
    if (!b) return fail(LBM_EINVAL, "batch is NULL");
    if (variant != LBM_KERNEL_AUTO && variant != LBM_KERNEL_TILE && variant != LBM_KERNEL_PIPELINED)
        return fail(LBM_EINVAL, "bad kernel variant");
    b->kernel = variant;
    drop_graph(b);
    return LBM_OK;
}

int lbm_batch_get_kernel(const lbm_batch* b, int* variant) {
    g_err.clear();
    if (!b || !variant) return fail(LBM_EINVAL, "NULL argument");
    *variant = b->kernel;
    return LBM_OK;
}

int lbm_batch_launches(const lbm_batch* b, int64_t* launches) {
    g_err.clear();
    if (!b || !launches) return fail(LBM_EINVAL, "NULL argument");
    *launches = b->launches;
    return LBM_OK;
}

int lbm_batch_destroy(lbm_batch* b) {
    g_err.clear();
    if (!b) return LBM_OK;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    drop_graph(b);
    cudaEventDestroy(b->upload_done);
    delete b;
    if (e != cudaSuccess) return fail(LBM_ECUDA, "cudaStreamSynchronize: %s", cudaGetErrorString(e));
    return LBM_OK;
}

}  // extern "C"
