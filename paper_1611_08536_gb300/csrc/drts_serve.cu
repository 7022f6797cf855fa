// Serving loop: continuous batching of independent DRTS simulations on one
// GPU.  Requests queue on the host; each tick
//   1. admits queued requests in arrival order while a resident slot and
//      device memory (a footprint estimate against the budget) are free,
//      assembling their A on the admission stream;
//   2. advances every resident simulation by up to steps_per_tick steps:
//      all their step launches are captured into one CUDA graph whose
//      branches fan out over n_streams streams, so the kernels of different
//      simulations overlap on the device, and the graph is launched once.
//      The executable graph is kept: a tick whose launches match the
//      previous one (same simulations and step counts, new parameters)
//      updates it in place instead of instantiating a new one;
//   3. retires finished simulations (detector history and ledger copied to
//      host, device memory freed), which frees room for the next admissions.
// Requests that arrive while others run are admitted at the next tick.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <exception>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "drts.h"
#include "drts_internal.h"

namespace drts {
cudaStream_t ctx_swap_stream(drts_ctx *c, cudaStream_t s);   // drts_api.cu
}

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id = 0;
    drts_problem prob{};
    std::vector<drts_medium> media;
    std::vector<uint8_t> mov;
    std::vector<int32_t> src_rhs;
    std::vector<int64_t> src_state;
    std::vector<double> src_w;
    int64_t t0 = 0;
    std::vector<double> profile;
    int64_t n_steps = 0;
    int32_t state = DRTS_REQ_QUEUED;
    drts_ctx *ctx = nullptr;
    int64_t footprint = 0;
    double work = 0.0;            // admission priority: voxels x 26 x passes per step x steps
    int32_t n_patch = 0;
    std::vector<double> det;      // [rhs][n_steps][n_patch]
    std::vector<double> ledger;   // [rhs][4]
    std::vector<double> final_x;  // [rhs][n_states] final states (keep_state only)
    Clock::time_point t_submit, t_admit, t_done;
    std::string error;
    // states per rhs held in final_x (0 when not kept)
    size_t state_n() const
    {
        return final_x.empty() ? 0 : final_x.size() / size_t(prob.n_rhs);
    }
};

}  // namespace

struct drts_server {
    drts_server_config cfg{};
    int64_t budget = 0, used = 0;
    int64_t next_id = 1;
    std::deque<int64_t> queue;
    std::vector<int64_t> resident;
    std::map<int64_t, std::unique_ptr<Request>> reqs;
    cudaStream_t main = nullptr, admit = nullptr;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev;
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t exec = nullptr;    // the tick graph, kept across ticks
    std::string err;
    drts_server_stats stats{};
};

namespace {

drts_status sfail(drts_server *s, drts_status st, const std::string &m)
{
    if (s) s->err = m;
    return st;
}

// The exception in flight at an entry point as a status (no C++ exception
// crosses the C ABI): DRTS_ENOMEM for a failed host allocation, else
// DRTS_EINVAL.  Call only from a catch handler.
drts_status scaught(drts_server *s, const char *where) noexcept
{
    drts_status st = DRTS_EINVAL;
    const char *what = "unknown exception";
    try {
        throw;
    } catch (const std::bad_alloc &) {
        st = DRTS_ENOMEM;
        what = "host allocation failed";
    } catch (const std::exception &ex) {
        what = ex.what();
    } catch (...) {
    }
    try {
        sfail(s, st, std::string(where) + ": " + what);
    } catch (...) {
    }
    return st;
}

// Device bytes a request will hold: the sliced matrix (about 220 stored
// slots per state with padding), two state buffers per right-hand side, the
// detector history and the per-voxel tables.
int64_t footprint_estimate(const drts_problem &p)
{
    const int64_t V = int64_t(p.nx) * p.ny * p.nz;
    const int64_t states = V * 26;
    const int64_t vb = p.precision == DRTS_FP64 ? 8 : (p.precision == DRTS_FP32 ? 4 : 2);
    const int64_t sb = p.precision == DRTS_FP64 ? 8 : 4;
    const int64_t n_patch = p.det_face >= 0 ? int64_t(p.det_nu) * p.det_nv : 0;
    // values + codes (FP16: a few large values per row stored as two terms)
    int64_t b = states * (p.precision == DRTS_FP16_ROWSCALE ? 225 : 220) * (vb + 2);
    const int64_t rhs_alloc = p.n_rhs == 1 ? 1 : (int64_t(p.n_rhs) + 3) / 4 * 4;   // groups of four
    b += 2 * (states + 64) * sb * rhs_alloc;                  // state ping-pong
    b += n_patch * p.max_steps * 8 * p.n_rhs;                 // detector history
    b += V * 2 + states * 4 + (states / 32) * 12 + (64 << 20);   // maps, row lengths, slice table, tables
    return b;
}

drts_status retire(drts_server *s, Request &r)
{
    drts_info info{};
    drts_get_info(r.ctx, &info);
    r.n_patch = info.n_patch;
    const int R = r.prob.n_rhs;
    r.det.assign(size_t(R) * r.n_steps * std::max(info.n_patch, 0), 0.0);
    r.ledger.assign(size_t(R) * 4, 0.0);
    drts_status st = DRTS_OK;
    if (s->cfg.keep_state) {
        r.final_x.assign(size_t(R) * size_t(info.n_states), 0.0);
        for (int q = 0; q < R && st == DRTS_OK; ++q)
            st = drts_read_state(r.ctx, q, r.final_x.data() + size_t(q) * size_t(info.n_states));
    }
    for (int q = 0; q < R && st == DRTS_OK; ++q)
        st = drts_read_detectors(r.ctx, q, 0, info.n_patch > 0 ? r.n_steps : 0,
                                 info.n_patch > 0 ? r.det.data() + size_t(q) * r.n_steps * info.n_patch : nullptr,
                                 r.ledger.data() + 4 * q);
    if (st != DRTS_OK) {
        r.error = drts_last_error(r.ctx);
        r.state = DRTS_REQ_FAILED;
        s->stats.failed++;
    } else {
        r.state = DRTS_REQ_DONE;
        s->stats.completed++;
    }
    drts_destroy(r.ctx);
    r.ctx = nullptr;
    s->used -= r.footprint;
    r.t_done = Clock::now();
    return st;
}

}  // namespace

extern "C" {

drts_status drts_server_create(const drts_server_config *cfg, drts_server **out)
try {
    if (!cfg || !out) return DRTS_EINVAL;
    *out = nullptr;
    if (cfg->max_resident < 1 || cfg->max_resident > 256 || cfg->steps_per_tick < 1 || cfg->n_streams < 1 ||
        cfg->n_streams > 32 || cfg->mem_budget_bytes < 0 || cfg->reserved != 0 ||
        (cfg->policy != DRTS_SERVE_FIFO && cfg->policy != DRTS_SERVE_SHORTEST_FIRST))
        return DRTS_EINVAL;
    std::unique_ptr<drts_server> s(new drts_server);
    s->cfg = *cfg;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return DRTS_ECUDA;
    s->budget = cfg->mem_budget_bytes ? cfg->mem_budget_bytes : int64_t(double(free_b) * 0.9);
    if (cudaStreamCreateWithFlags(&s->main, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->admit, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming) != cudaSuccess)
        return DRTS_ECUDA;
    s->side.resize(cfg->n_streams);
    s->ev.resize(cfg->n_streams);
    for (int i = 0; i < cfg->n_streams; ++i)
        if (cudaStreamCreateWithFlags(&s->side[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s->ev[i], cudaEventDisableTiming) != cudaSuccess)
            return DRTS_ECUDA;
    *out = s.release();
    return DRTS_OK;
} catch (...) {
    return scaught(nullptr, "drts_server_create");
}

drts_status drts_server_submit(drts_server *s, const drts_problem *prob, int32_t n_entries, const int32_t *src_rhs,
                               const int64_t *src_state, const double *src_weight, int64_t t0, int32_t n_t,
                               const double *profile, int64_t n_steps, int64_t *request_id)
try {
    if (!s || !prob || !request_id) return DRTS_EINVAL;
    if (n_steps < 1) return sfail(s, DRTS_EINVAL, "n_steps must be >= 1");
    if (!prob->media || !prob->medium_of_voxel || prob->n_media < 1 || prob->nx < 2 || prob->ny < 2 || prob->nz < 2)
        return sfail(s, DRTS_EINVAL, "incomplete problem");
    if (n_entries < 0 || (n_entries > 0 && (!src_rhs || !src_state || !src_weight)) || n_t < 0 ||
        (n_t > 0 && !profile))
        return sfail(s, DRTS_EINVAL, "bad sources");
    std::unique_ptr<Request> r(new Request);
    r->id = s->next_id++;
    r->prob = *prob;
    r->prob.max_steps = n_steps;
    r->media.assign(prob->media, prob->media + prob->n_media);
    const int64_t V = int64_t(prob->nx) * prob->ny * prob->nz;
    r->mov.assign(prob->medium_of_voxel, prob->medium_of_voxel + V);
    r->prob.media = r->media.data();
    r->prob.medium_of_voxel = r->mov.data();
    r->src_rhs.assign(src_rhs, src_rhs + n_entries);
    r->src_state.assign(src_state, src_state + n_entries);
    r->src_w.assign(src_weight, src_weight + n_entries);
    for (int32_t q : r->src_rhs)
        if (q < 0 || q >= prob->n_rhs) return sfail(s, DRTS_EINVAL, "source rhs out of range");
    r->t0 = t0;
    r->profile.assign(profile, profile + n_t);
    r->n_steps = n_steps;
    r->footprint = footprint_estimate(r->prob);
    // one pass over A per 8 right-hand sides (the batched step's default tile)
    r->work = double(V) * 26.0 * double((prob->n_rhs + 7) / 8) * double(n_steps);
    if (r->footprint > s->budget) return sfail(s, DRTS_ENOMEM, "request larger than the memory budget");
    r->t_submit = Clock::now();
    *request_id = r->id;
    s->queue.push_back(r->id);
    s->reqs[r->id] = std::move(r);
    s->stats.submitted++;
    return DRTS_OK;
} catch (...) {
    return scaught(s, "drts_server_submit");
}

drts_status drts_server_tick(drts_server *s, int32_t *n_done)
try {
    drts::NvtxRange nvtx("drts_server_tick");
    if (!s) return DRTS_EINVAL;
    int32_t done = 0;
    // 1. the steps of every resident simulation, captured in one graph
    std::vector<int64_t> running;
    for (int64_t id : s->resident) running.push_back(id);
    if (!running.empty()) {
        const Clock::time_point t_graph = Clock::now();
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s->main, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = cudaEventRecord(s->fork, s->main);
        for (int i = 0; i < s->cfg.n_streams && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(s->side[i], s->fork, 0);
        drts_status st = DRTS_OK;
        for (size_t k = 0; k < running.size() && e == cudaSuccess && st == DRTS_OK; ++k) {
            Request &r = *s->reqs[running[k]];
            drts_info info{};
            drts_get_info(r.ctx, &info);
            const int64_t n = std::min<int64_t>(s->cfg.steps_per_tick, r.n_steps - info.t);
            cudaStream_t old = drts::ctx_swap_stream(r.ctx, s->side[k % s->cfg.n_streams]);
            st = drts_step_n(r.ctx, n);
            drts::ctx_swap_stream(r.ctx, old);
        }
        for (int i = 0; i < s->cfg.n_streams && e == cudaSuccess; ++i) {
            e = cudaEventRecord(s->ev[i], s->side[i]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s->main, s->ev[i], 0);
        }
        cudaError_t e2 = cudaStreamEndCapture(s->main, &graph);
        if (e == cudaSuccess) e = e2;
        if (st != DRTS_OK) {
            if (graph) cudaGraphDestroy(graph);
            return sfail(s, st, "tick: step launch failed during capture");
        }
        // the previous tick's executable graph takes the new parameters when
        // the launches are the same (same simulations, same step counts);
        // otherwise a new one is instantiated
        if (e == cudaSuccess && s->exec) {
            cudaGraphExecUpdateResultInfo ui{};
            if (cudaGraphExecUpdate(s->exec, graph, &ui) == cudaSuccess) {
                s->stats.graph_updates++;
            } else {
                cudaGetLastError();
                cudaGraphExecDestroy(s->exec);
                s->exec = nullptr;
            }
        }
        bool instantiated = false;
        if (e == cudaSuccess && !s->exec) {
            e = cudaGraphInstantiate(&s->exec, graph, 0);
            if (e == cudaSuccess) s->stats.graph_instantiations++;
            else s->exec = nullptr;
            instantiated = true;
        }
        if (graph) cudaGraphDestroy(graph);
        const double host_s = std::chrono::duration<double>(Clock::now() - t_graph).count();
        s->stats.host_graph_s += host_s;
        if (instantiated) s->stats.host_instantiate_s += host_s;
        if (e == cudaSuccess) e = cudaGraphLaunch(s->exec, s->main);
        if (e != cudaSuccess) {
            if (s->exec) cudaGraphExecDestroy(s->exec);
            s->exec = nullptr;
            return sfail(s, DRTS_ECUDA, std::string("tick graph: ") + cudaGetErrorString(e));
        }
        s->stats.ticks++;
        s->stats.graph_launches++;
    }
    // 2. admissions overlap the tick on the admission stream
    while (!s->queue.empty() && int(s->resident.size()) < s->cfg.max_resident) {
        auto pick = s->queue.begin();
        if (s->cfg.policy == DRTS_SERVE_SHORTEST_FIRST)
            for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
                if (s->reqs[*it]->work < s->reqs[*pick]->work) pick = it;
        Request &r = *s->reqs[*pick];
        if (s->used + r.footprint > s->budget) break;
        drts_ctx *ctx = nullptr;
        drts_status st = drts_assemble(&r.prob, s->admit, &ctx);
        if (st == DRTS_OK) {
            for (int q = 0; q < r.prob.n_rhs && st == DRTS_OK; ++q) {
                std::vector<int64_t> stq;
                std::vector<double> wq;
                for (size_t e = 0; e < r.src_rhs.size(); ++e)
                    if (r.src_rhs[e] == q) {
                        stq.push_back(r.src_state[e]);
                        wq.push_back(r.src_w[e]);
                    }
                st = drts_inject_source(ctx, q, int32_t(stq.size()), stq.data(), wq.data(), r.t0,
                                        int32_t(r.profile.size()), r.profile.data());
            }
        }
        s->queue.erase(pick);
        if (st != DRTS_OK) {
            r.error = ctx ? drts_last_error(ctx) : drts_last_error(nullptr);
            if (ctx) drts_destroy(ctx);
            r.state = DRTS_REQ_FAILED;
            r.t_done = Clock::now();
            s->stats.failed++;
            continue;
        }
        drts::ctx_swap_stream(ctx, s->main);
        r.ctx = ctx;
        r.state = DRTS_REQ_RUNNING;
        r.t_admit = Clock::now();
        s->used += r.footprint;
        s->resident.push_back(r.id);
        s->stats.admitted++;
    }
    // 3. wait for the tick, retire finished simulations
    cudaError_t e = cudaStreamSynchronize(s->main);
    if (e != cudaSuccess) return sfail(s, DRTS_ECUDA, std::string("tick: ") + cudaGetErrorString(e));
    std::vector<int64_t> keep;
    for (int64_t id : running) {
        Request &r = *s->reqs[id];
        drts_info info{};
        drts_get_info(r.ctx, &info);
        if (info.t >= r.n_steps) {
            retire(s, r);
            ++done;
        } else {
            keep.push_back(id);
        }
    }
    for (int64_t id : s->resident)
        if (std::find(running.begin(), running.end(), id) == running.end()) keep.push_back(id);
    s->resident = keep;
    s->stats.resident = int32_t(s->resident.size());
    s->stats.queued = int32_t(s->queue.size());
    s->stats.used_bytes = s->used;
    if (n_done) *n_done = done;
    return DRTS_OK;
} catch (...) {
    return scaught(s, "drts_server_tick");
}

drts_status drts_server_poll(drts_server *s, int64_t id, drts_request_info *out)
try {
    if (!s || !out) return DRTS_EINVAL;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, DRTS_EINVAL, "unknown request");
    const Request &r = *it->second;
    std::memset(out, 0, sizeof(*out));
    out->state = r.state;
    out->n_steps = r.n_steps;
    out->n_rhs = r.prob.n_rhs;
    out->n_patch = r.n_patch;
    out->footprint_bytes = r.footprint;
    auto secs = [&](Clock::time_point a, Clock::time_point b) {
        return std::chrono::duration<double>(b - a).count();
    };
    if (r.state == DRTS_REQ_RUNNING || r.state == DRTS_REQ_DONE) out->queue_s = secs(r.t_submit, r.t_admit);
    if (r.state == DRTS_REQ_DONE || r.state == DRTS_REQ_FAILED) out->latency_s = secs(r.t_submit, r.t_done);
    return DRTS_OK;
} catch (...) {
    return scaught(s, "drts_server_poll");
}

drts_status drts_server_result(drts_server *s, int64_t id, int32_t rhs, double *det_out, double *ledger_out)
try {
    if (!s) return DRTS_EINVAL;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, DRTS_EINVAL, "unknown request");
    const Request &r = *it->second;
    if (r.state != DRTS_REQ_DONE) return sfail(s, DRTS_ESTATE, r.error.empty() ? "request not done" : r.error);
    if (rhs < 0 || rhs >= r.prob.n_rhs) return sfail(s, DRTS_EINVAL, "rhs out of range");
    if (det_out && r.n_patch > 0)
        std::memcpy(det_out, r.det.data() + size_t(rhs) * r.n_steps * r.n_patch,
                    sizeof(double) * r.n_steps * r.n_patch);
    if (ledger_out) std::memcpy(ledger_out, r.ledger.data() + 4 * rhs, 4 * sizeof(double));
    return DRTS_OK;
} catch (...) {
    return scaught(s, "drts_server_result");
}

drts_status drts_server_result_state(drts_server *s, int64_t id, int32_t rhs, double *state_out)
try {
    if (!s) return DRTS_EINVAL;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, DRTS_EINVAL, "unknown request");
    const Request &r = *it->second;
    if (r.state != DRTS_REQ_DONE) return sfail(s, DRTS_ESTATE, r.error.empty() ? "request not done" : r.error);
    if (rhs < 0 || rhs >= r.prob.n_rhs || !state_out) return sfail(s, DRTS_EINVAL, "bad rhs or NULL buffer");
    if (r.state_n() == 0) return sfail(s, DRTS_ESTATE, "final states are kept only with keep_state");
    const size_t n = r.state_n();
    std::memcpy(state_out, r.final_x.data() + size_t(rhs) * n, n * sizeof(double));
    return DRTS_OK;
} catch (...) {
    return scaught(s, "drts_server_result_state");
}

drts_status drts_server_cancel(drts_server *s, int64_t id)
try {
    if (!s) return DRTS_EINVAL;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, DRTS_EINVAL, "unknown request");
    Request &r = *it->second;
    if (r.state == DRTS_REQ_QUEUED) {
        auto q = std::find(s->queue.begin(), s->queue.end(), id);
        if (q != s->queue.end()) s->queue.erase(q);
    } else if (r.state == DRTS_REQ_RUNNING) {
        // between ticks; the tick graph joins every side stream back into
        // the main stream, so these two waits leave nothing in flight
        cudaError_t e = cudaStreamSynchronize(s->main);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->admit);
        if (e != cudaSuccess) return sfail(s, DRTS_ECUDA, std::string("cancel: ") + cudaGetErrorString(e));
        drts_destroy(r.ctx);
        r.ctx = nullptr;
        s->used -= r.footprint;
        auto k = std::find(s->resident.begin(), s->resident.end(), id);
        if (k != s->resident.end()) s->resident.erase(k);
    } else {
        return sfail(s, DRTS_ESTATE, "request already finished, failed or cancelled");
    }
    r.state = DRTS_REQ_CANCELLED;
    r.error = "request cancelled";
    r.t_done = Clock::now();
    s->stats.cancelled++;
    return DRTS_OK;
} catch (...) {
    return scaught(s, "drts_server_cancel");
}

drts_status drts_server_release(drts_server *s, int64_t id)
try {
    if (!s) return DRTS_EINVAL;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, DRTS_EINVAL, "unknown request");
    if (it->second->state == DRTS_REQ_QUEUED || it->second->state == DRTS_REQ_RUNNING)
        return sfail(s, DRTS_ESTATE, "request still queued or running");
    s->reqs.erase(it);
    return DRTS_OK;
} catch (...) {
    return scaught(s, "drts_server_release");
}

drts_status drts_server_get_stats(const drts_server *s, drts_server_stats *out)
{
    if (!s || !out) return DRTS_EINVAL;
    *out = s->stats;
    out->resident = int32_t(s->resident.size());     // live counts, not the last tick's
    out->queued = int32_t(s->queue.size());
    out->used_bytes = s->used;
    out->budget_bytes = s->budget;
    return DRTS_OK;
}

const char *drts_server_last_error(const drts_server *s)
{
    return s ? s->err.c_str() : "";
}

void drts_server_destroy(drts_server *s)
{
    if (!s) return;
    cudaStreamSynchronize(s->main);
    cudaStreamSynchronize(s->admit);
    for (auto &kv : s->reqs)
        if (kv.second->ctx) drts_destroy(kv.second->ctx);
    for (size_t i = 0; i < s->side.size(); ++i) {
        cudaStreamDestroy(s->side[i]);
        cudaEventDestroy(s->ev[i]);
    }
    cudaEventDestroy(s->fork);
    if (s->exec) cudaGraphExecDestroy(s->exec);
    cudaStreamDestroy(s->main);
    cudaStreamDestroy(s->admit);
    delete s;
}

}  // extern "C"
