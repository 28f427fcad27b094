// rve_plan.cu -- plans (the whole pipeline of a fixed batch captured once in
// a CUDA graph and relaunched) and the tile-shape autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "rve_common.cuh"
#include "rve_internal.h"

namespace rve {

// ------------------------------------------------------------ tuner table --
// (n, precision, path) -> (stencil tile rows, column-block threads).
static std::mutex g_tune_lock;
static std::map<std::tuple<int, int, int>, std::pair<int, int>> g_tune;

bool tuned_tiles(int n, int precision, int path, int* tS, int* blockC) {
    std::lock_guard<std::mutex> g(g_tune_lock);
    auto it = g_tune.find(std::make_tuple(n, precision, path));
    if (it == g_tune.end()) return false;
    *tS = it->second.first;
    *blockC = it->second.second;
    return true;
}

static void set_tuned(int n, int precision, int path, int tS, int blockC) {
    std::lock_guard<std::mutex> g(g_tune_lock);
    g_tune[std::make_tuple(n, precision, path)] = std::make_pair(tS, blockC);
}

// Pipeline of one batch into the stream: field, solve (persistent path),
// A_hom.  Buffers are carved from ws: [mask | u | solver workspace].
struct PipeLayout {
    size_t o_mask, o_u, o_info, o_solve, total;
};

static PipeLayout pipe_layout(const Plan& p) {
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    PipeLayout l;
    l.o_mask = 0;
    l.o_u = up(sizeof(uint32_t) * (size_t)p.words);
    l.o_info = l.o_u + up(sizeof(double) * 2 * (size_t)p.nodes);
    l.o_solve = l.o_info + up(sizeof(rve_solve_info) * (size_t)p.batch);
    l.total = l.o_solve + p.total;
    return l;
}

}  // namespace rve

using namespace rve;

struct rve_plan_s {
    Plan p;
    rve_solve_opts o;
    PipeLayout l;
    cudaGraphExec_t exec = nullptr;
    void* ws = nullptr;
    double* A = nullptr;
    rve_solve_info* info = nullptr;
    int kernels = 0;   // kernel nodes of the captured graph (launch diagnostics)
};

extern "C" {

rve_status rve_plan_create(const rve_realization* r, int32_t batch, const rve_solve_opts* opts,
                           rve_plan* out) {
    if (!out) return RVE_EINVAL;
    *out = nullptr;
    rve_solve_opts o = {};
    if (opts) o = *opts;
    // graph-capturable paths only (no host synchronisation): the persistent
    // kernel, or the fused kernels inside a conditional while node
    if (o.path == RVE_PATH_PLAIN) return RVE_EINVAL;
    rve_plan_s* pl = new rve_plan_s();
    rve_status st = make_plan(r, batch, &o, pl->p, true);
    if (st != RVE_OK) {
        delete pl;
        return st;
    }
    pl->o = resolved_opts(&o);
    pl->l = pipe_layout(pl->p);
    *out = pl;
    return RVE_OK;
}

size_t rve_plan_workspace_size(rve_plan plan) { return plan ? plan->l.total : 0; }

rve_status rve_plan_execute(rve_plan plan, double* A, rve_solve_info* info, void* ws,
                            size_t ws_bytes, void* stream) {
    // a graph cannot be captured on the legacy default stream
    if (!plan || !A || !info || !ws || ws_misaligned(ws) || !stream) return RVE_EINVAL;
    if (ws_bytes < plan->l.total) return RVE_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!plan->exec || plan->ws != ws || plan->A != A || plan->info != info) {
        if (plan->exec) {
            cudaGraphExecDestroy(plan->exec);
            plan->exec = nullptr;
        }
        const Plan& p = plan->p;
        char* w = static_cast<char*>(ws);
        uint32_t* mask = reinterpret_cast<uint32_t*>(w + plan->l.o_mask);
        double* u = reinterpret_cast<double*>(w + plan->l.o_u);
        void* sw = w + plan->l.o_solve;
        // descriptors (pageable host -> device) and kernel attributes before
        // the capture; everything captured is a kernel or a memset
        if (upload_descriptors(p, sw, s) != RVE_OK || cudaStreamSynchronize(s) != cudaSuccess)
            return note_error("plan: descriptor upload", cudaGetLastError());
        const bool loop = plan->p.path == RVE_PATH_FUSED;
        if ((loop ? prepare_graph_loop(plan->p) : prepare_persistent(plan->p)) != RVE_OK)
            return note_error("plan: kernel set-up", cudaGetLastError());
        cudaGraph_t graph = nullptr;
        const long long noted = g_launches.load();
        cudaError_t be = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (be != cudaSuccess) return note_error("plan: begin capture", be);
        rve_status st = RVE_OK;
        if (launch_gen_field(p, nullptr, mask, s) != cudaSuccess) st = RVE_ECUDA;
        if (st == RVE_OK)
            st = loop ? enqueue_solve_graph_loop(p, sw, mask, nullptr, plan->o, u, info, s)
                      : enqueue_solve_persistent(p, sw, mask, nullptr, plan->o, u, info, s);
        if (st == RVE_OK &&
            launch_a_hom(p, sw, mask, nullptr, p.scheme, p.precision, u, A, nullptr, nullptr, s) != cudaSuccess)
            st = RVE_ECUDA;
        const cudaError_t le = cudaGetLastError();
        const cudaError_t ce = cudaStreamEndCapture(s, &graph);
        // the launches noted while capturing were recorded, not run: they are
        // counted each time the graph runs instead
        plan->kernels = (int)(g_launches.load() - noted);
        g_launches.fetch_sub(plan->kernels);
        if (st != RVE_OK || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return note_error("plan: capture", ce != cudaSuccess ? ce : le);
        }
        const cudaError_t ie = cudaGraphInstantiate(&plan->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            plan->exec = nullptr;
            return note_error("plan: instantiate", ie);
        }
        plan->ws = ws;
        plan->A = A;
        plan->info = info;
    }
    note_launch(plan->kernels);
    const cudaError_t ge = cudaGraphLaunch(plan->exec, s);
    return ge == cudaSuccess ? RVE_OK : note_error("plan: graph launch", ge);
}

void rve_plan_destroy(rve_plan plan) {
    if (!plan) return;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    delete plan;
}

// ------------------------------------------------------------------ tuner --
rve_status rve_autotune(const rve_realization* r, int32_t batch, const rve_solve_opts* opts,
                        void* ws, size_t ws_bytes, void* stream) {
    Plan all;
    rve_status st = make_plan(r, batch, opts, all, false);
    if (st != RVE_OK) return st;
    if (!ws || ws_misaligned(ws)) return RVE_EINVAL;
    const rve_solve_opts base = resolved_opts(opts);
    if (base.path == RVE_PATH_PLAIN) return RVE_OK;   // nothing to tune
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return RVE_ECUDA;
    std::vector<int> sizes;
    for (int b = 0; b < batch; ++b) {
        const int n = r[b].L * r[b].m0;
        if (std::find(sizes.begin(), sizes.end(), n) == sizes.end()) sizes.push_back(n);
    }
    st = RVE_OK;
    for (int n : sizes) {
        std::vector<rve_realization> sub;
        for (int b = 0; b < batch && (int)sub.size() < 16; ++b)
            if (r[b].L * r[b].m0 == n) sub.push_back(r[b]);
        // stencil tile heights: tS + 2 a multiple of the transform group
        // G = 2048/n (no idle row slots), plus a few small powers of two
        std::vector<int> tss;
        const int G = std::max(1, 2048 / n);
        for (int k = 1; k <= 4; ++k) tss.push_back(std::min(k * G - 2, n));
        for (int v : {2, 4, 8}) tss.push_back(v);
        std::sort(tss.begin(), tss.end());
        tss.erase(std::unique(tss.begin(), tss.end()), tss.end());
        tss.erase(std::remove_if(tss.begin(), tss.end(), [&](int v) { return v < 1 || v > n; }),
                  tss.end());
        std::vector<int> bcs = {128, 256, 512};
        if (base.path == RVE_PATH_PERSISTENT) bcs = {256};
        float best = 1e30f;
        int best_ts = 0, best_bc = 0;
        for (int ts : tss) {
            for (int bc : bcs) {
                if (ts > n) continue;
                rve_solve_opts o = base;
                o.tile_rows = ts;
                o.col_tile = bc;
                o.max_iter = 12;   // a short trial: the time is that of iteration steps
                Plan p;
                if (make_plan(sub.data(), (int)sub.size(), &o, p, true) != RVE_OK) continue;
                const PipeLayout l = pipe_layout(p);
                if (l.total > ws_bytes) continue;
                char* w = static_cast<char*>(ws);
                uint32_t* mask = reinterpret_cast<uint32_t*>(w + l.o_mask);
                double* u = reinterpret_cast<double*>(w + l.o_u);
                rve_solve_info* inf = reinterpret_cast<rve_solve_info*>(w + l.o_info);
                if (launch_gen_field(p, nullptr, mask, s) != cudaSuccess) { st = RVE_ECUDA; break; }
                float t = 1e30f;
                for (int rep = 0; rep < 2; ++rep) {
                    cudaEventRecord(e0, s);
                    rve_status rs = RVE_OK;
                    if (o.path == RVE_PATH_PERSISTENT) {
                        rs = prepare_persistent(p);
                        if (rs == RVE_OK)
                            rs = run_solve_persistent(p, w + l.o_solve, mask, nullptr, o, u, inf, s);
                    } else {
                        rs = run_solve_fused(p, w + l.o_solve, mask, nullptr, o, u, inf, s);
                    }
                    cudaEventRecord(e1, s);
                    if (rs != RVE_OK || cudaEventSynchronize(e1) != cudaSuccess) {
                        st = RVE_ECUDA;
                        break;
                    }
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    t = std::min(t, ms);
                }
                if (st != RVE_OK) break;
                if (t < best) {
                    best = t;
                    best_ts = ts;
                    best_bc = bc;
                }
            }
            if (st != RVE_OK) break;
        }
        if (st != RVE_OK) break;
        if (best_ts > 0)
            set_tuned(n, base.precision, base.path == RVE_PATH_PERSISTENT ? 1 : 0, best_ts, best_bc);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

rve_status rve_tuner_save(const char* path) {
    if (!path) return RVE_EINVAL;
    FILE* f = std::fopen(path, "w");
    if (!f) return RVE_EINVAL;
    std::lock_guard<std::mutex> g(g_tune_lock);
    std::fprintf(f, "# n precision persistent tile_rows block_threads\n");
    for (const auto& kv : g_tune)
        std::fprintf(f, "%d %d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first),
                     std::get<2>(kv.first), kv.second.first, kv.second.second);
    std::fclose(f);
    return RVE_OK;
}

rve_status rve_tuner_load(const char* path) {
    if (!path) return RVE_EINVAL;
    FILE* f = std::fopen(path, "r");
    if (!f) return RVE_EINVAL;
    char line[256];
    while (std::fgets(line, sizeof line, f)) {
        if (line[0] == '#') continue;
        int n, pr, pe, ts, bc;
        if (std::sscanf(line, "%d %d %d %d %d", &n, &pr, &pe, &ts, &bc) == 5)
            set_tuned(n, pr, pe, ts, bc);
    }
    std::fclose(f);
    return RVE_OK;
}

int32_t rve_tuner_lookup(int32_t n, int32_t precision, int32_t persistent, int32_t* tile_rows,
                         int32_t* block_threads) {
    int ts = 0, bc = 0;
    if (!tuned_tiles(n, precision, persistent ? 1 : 0, &ts, &bc)) return 0;
    if (tile_rows) *tile_rows = ts;
    if (block_threads) *block_threads = bc;
    return 1;
}

void rve_tuner_clear(void) {
    std::lock_guard<std::mutex> g(g_tune_lock);
    g_tune.clear();
}

}  // extern "C"
