// cfpq_server.cu -- continuous-batching query server over a resident graph.
//
// Each submitted RSM becomes a query with its own device state (closure
// blocks, M2/A2, loop control).  A step admits waiting queries whose planned
// device footprint fits the memory budget (first come, first served), runs a
// few fixpoint passes for every running query in shared launches (the same
// executor as cfpq_batch_run), and retires the queries whose loop finished.
// Queries therefore join and leave the running set between passes while the
// others keep their state on the device.
#include <chrono>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "cfpq_engine.cuh"

using namespace cfpq;

namespace {
constexpr uint32_t kServerPassCap = 1u << 20;
constexpr uint32_t kPassesPerStep = 8;
enum JobState { kWaiting = 0, kRunning = 1, kDone = 2, kFailed = 3 };
}  // namespace

struct cfpq_server {
    cfpq_options opt;
    cudaStream_t stream = nullptr;
    Allocator A;
    std::string err;
    GraphDev graph;
    struct Job {
        uint64_t ticket = 0;
        int state = kWaiting;
        int status = CFPQ_OK;
        std::unique_ptr<QueryDev> q;
        QCtl final_ctl;
    };
    std::map<uint64_t, Job> jobs;
    std::deque<uint64_t> waiting;
    std::vector<uint64_t> running;
    Executor exec;
    bool exec_dirty = true;
    uint64_t next_ticket = 1;
    size_t budget = 0;
};

namespace {
int sfail(cfpq_server *s, int code, const std::string &m) {
    if (s) s->err = m;
    return code;
}
#define SCK(s, call)                                                                                  \
    do {                                                                                              \
        cudaError_t _e = (call);                                                                      \
        if (_e != cudaSuccess) return sfail(s, CFPQ_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
    } while (0)
}  // namespace

extern "C" {

int cfpq_server_create(cfpq_server **out, const cfpq_options *opt, void *stream, uint32_t n_vertices,
                       uint32_t n_terminals, size_t n_edges, const uint32_t *src, const uint32_t *label,
                       const uint32_t *dst) {
    if (!out) return CFPQ_ERR_INVALID_ARG;
    *out = nullptr;
    try {
        std::unique_ptr<cfpq_server> s(new cfpq_server());
        if (opt) {
            if (opt->struct_size != sizeof(cfpq_options)) return CFPQ_ERR_INVALID_ARG;
            s->opt = *opt;
        } else {
            cfpq_default_options(&s->opt);
        }
        if ((s->opt.alloc == nullptr) != (s->opt.free == nullptr)) return CFPQ_ERR_INVALID_ARG;
        if (s->opt.closure_mode > CFPQ_CLOSURE_TC_FP4 || s->opt.tile_format > CFPQ_TILES_NVFP4)
            return CFPQ_ERR_INVALID_ARG;
        if (s->opt.closure_mode == CFPQ_CLOSURE_TC_I8) return CFPQ_ERR_UNSUPPORTED;
        if (cudaSetDevice(s->opt.device) != cudaSuccess) {
            cudaGetLastError();
            return CFPQ_ERR_CUDA;
        }
        s->stream = static_cast<cudaStream_t>(stream);
        s->A.alloc = s->opt.alloc;
        s->A.free = s->opt.free;
        s->A.user = s->opt.alloc_user;
        s->A.stream = s->stream;
        // work items of 4x the rows: the running set changes (and the work
        // lists are re-assembled on the host) at most every step, and the
        // assembly's cost grows with the number of items
        s->exec.item_scale = 4;
        std::string e;
        int rc = stage_graph(&s->graph, &s->A, s->stream, n_vertices, n_terminals, n_edges, src, label, dst, false, &e);
        if (rc) return rc;
        if (s->opt.memory_budget) {
            s->budget = s->opt.memory_budget;
        } else {
            size_t fr = 0, tot = 0;
            if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return CFPQ_ERR_CUDA;
            const size_t margin = (size_t)2 << 30;
            s->budget = s->A.in_use + (fr > margin ? fr - margin : fr / 2);
        }
        *out = s.release();
        return CFPQ_OK;
    } catch (...) {
        return CFPQ_ERR_OUT_OF_MEMORY;
    }
}

int cfpq_server_destroy(cfpq_server *s) {
    if (!s) return CFPQ_OK;
    cudaSetDevice(s->opt.device);
    cudaStreamSynchronize(s->stream);
    delete s;
    return CFPQ_OK;
}

int cfpq_submit(cfpq_server *s, const cfpq_rsm *rsm, uint64_t *ticket) {
    if (!s || !ticket) return CFPQ_ERR_INVALID_ARG;
    try {
        cfpq_server::Job j;
        j.q.reset(new QueryDev());
        // AUTO serves with bit-packed rows only: tile products would add an
        // n x n-byte operand workspace per dense source to every query's
        // footprint and cut the number of queries admitted together
        j.q->closure_mode = s->opt.closure_mode == CFPQ_CLOSURE_AUTO ? (uint32_t)CFPQ_CLOSURE_BITPACKED
                                                                     : s->opt.closure_mode;
        {
            cfpq_options o = s->opt;
            o.closure_mode = j.q->closure_mode;
            set_tiles(*j.q, o, s->stream, s->graph.n);
        }
        j.q->gather_slices = s->opt.gather_slices;
        std::string e;
        int rc = copy_rsm(rsm, &j.q->rsm, &e);
        if (rc) return sfail(s, rc, e);
        j.q->g = &s->graph;
        rc = j.q->plan(&e);
        if (rc) return sfail(s, rc, e);
        j.ticket = s->next_ticket++;
        *ticket = j.ticket;
        s->waiting.push_back(j.ticket);
        s->jobs.emplace(j.ticket, std::move(j));
        return CFPQ_OK;
    } catch (...) {
        return sfail(s, CFPQ_ERR_OUT_OF_MEMORY, "host allocation failed");
    }
}

int cfpq_server_step(cfpq_server *s, uint32_t *n_running, uint32_t *n_waiting) {
    if (!s) return CFPQ_ERR_INVALID_ARG;
    try {
        SCK(s, cudaSetDevice(s->opt.device));
        std::string e;
        // 1. admission by planned device footprint, first come first served
        while (!s->waiting.empty()) {
            auto &j = s->jobs[s->waiting.front()];
            const uint64_t need = j.q->footprint();
            if (need > s->budget) {
                j.state = kFailed;
                j.status = CFPQ_ERR_OUT_OF_MEMORY;
                s->waiting.pop_front();
                continue;
            }
            if (s->A.in_use + need > s->budget) break;
            int rc = j.q->prepare(&s->A, &e);
            if (rc == CFPQ_ERR_OUT_OF_MEMORY && !s->running.empty()) break;  // wait for memory
            if (rc) {
                j.state = kFailed;
                j.status = rc;
                s->waiting.pop_front();
                continue;
            }
            rc = j.q->enqueue_init(s->stream, s->opt.max_iterations, s->opt.max_rounds, kServerPassCap);
            if (rc) return sfail(s, rc, "query initialisation failed");
            j.state = kRunning;
            s->running.push_back(j.ticket);
            s->waiting.pop_front();
            s->exec_dirty = true;
        }
        // 2. passes for every running query
        if (!s->running.empty()) {
            if (s->exec_dirty) {
                s->exec.qs.clear();
                for (uint64_t t : s->running) s->exec.qs.push_back(s->jobs[t].q.get());
                int rc = s->exec.assemble(&s->A, s->stream, &e);
                if (rc) return sfail(s, rc, e);
                if (s->exec.enqueue_lists(s->stream)) return sfail(s, CFPQ_ERR_CUDA, "list launch failed");
                s->exec_dirty = false;
            }
            for (uint32_t p = 0; p < kPassesPerStep; ++p)
                if (s->exec.enqueue_pass(s->stream, 0, 0, nullptr)) return sfail(s, CFPQ_ERR_CUDA, "pass launch failed");
            std::vector<QCtl> ctls;
            if (s->exec.read_ctls(s->stream, &ctls)) return sfail(s, CFPQ_ERR_CUDA, "reading loop state failed");
            // 3. retire finished queries
            std::vector<uint64_t> still;
            for (size_t i = 0; i < s->running.size(); ++i) {
                auto &j = s->jobs[s->running[i]];
                if (ctls[i].phase == kPhaseDone) {
                    j.state = kDone;
                    j.final_ctl = ctls[i];
                    j.status = ctls[i].status == kStatusOk ? CFPQ_OK : CFPQ_ERR_TIMEOUT;
                    s->exec_dirty = true;
                } else {
                    still.push_back(s->running[i]);
                }
            }
            s->running.swap(still);
        }
        if (n_running) *n_running = (uint32_t)s->running.size();
        if (n_waiting) *n_waiting = (uint32_t)s->waiting.size();
        return CFPQ_OK;
    } catch (...) {
        return sfail(s, CFPQ_ERR_OUT_OF_MEMORY, "host allocation failed");
    }
}

int cfpq_poll(cfpq_server *s, uint64_t ticket, int *done) {
    if (!s || !done) return CFPQ_ERR_INVALID_ARG;
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return sfail(s, CFPQ_ERR_INVALID_ARG, "unknown ticket");
    *done = (it->second.state == kDone || it->second.state == kFailed) ? 1 : 0;
    return it->second.state == kFailed ? it->second.status : CFPQ_OK;
}

int cfpq_result_reachable_bits(cfpq_server *s, uint64_t ticket, uint32_t box, uint64_t *bits) {
    if (!s || !bits) return CFPQ_ERR_INVALID_ARG;
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return sfail(s, CFPQ_ERR_INVALID_ARG, "unknown ticket");
    auto &j = it->second;
    if (j.state == kFailed) return j.status;
    if (j.state != kDone) return sfail(s, CFPQ_ERR_NOT_READY, "query not finished");
    if (box >= j.q->B) return sfail(s, CFPQ_ERR_INVALID_ARG, "box out of range");
    SCK(s, cudaSetDevice(s->opt.device));
    const size_t wn = (j.q->n + 63) / 64;
    SCK(s, cudaMemcpy2DAsync(bits, wn * 8, j.q->m2_ptr(box), (size_t)j.q->W * 8, wn * 8, j.q->n,
                             cudaMemcpyDeviceToHost, s->stream));
    SCK(s, cudaStreamSynchronize(s->stream));
    return j.status;
}

int cfpq_release(cfpq_server *s, uint64_t ticket) {
    if (!s) return CFPQ_ERR_INVALID_ARG;
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return sfail(s, CFPQ_ERR_INVALID_ARG, "unknown ticket");
    if (it->second.state == kRunning) {
        // cancelled: its passes run only inside cfpq_server_step, which
        // returns with the stream drained, so nothing of it is in flight;
        // the next step assembles the work lists without it
        for (auto r = s->running.begin(); r != s->running.end(); ++r)
            if (*r == ticket) {
                s->running.erase(r);
                break;
            }
        s->exec_dirty = true;
        if (cudaSetDevice(s->opt.device) != cudaSuccess || cudaStreamSynchronize(s->stream) != cudaSuccess)
            return sfail(s, CFPQ_ERR_CUDA, "stream synchronisation failed");
    }
    if (it->second.state == kWaiting) {
        for (auto w = s->waiting.begin(); w != s->waiting.end(); ++w)
            if (*w == ticket) {
                s->waiting.erase(w);
                break;
            }
    }
    cudaSetDevice(s->opt.device);
    s->jobs.erase(it);
    return CFPQ_OK;
}

}  // extern "C"
