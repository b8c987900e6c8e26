// qaoa_server.cu -- serving loop of libqaoa: continuous batching of optimise-and-sample jobs.
//
// A job is one sub-QUBO (n, p, Q, initial parameters) that runs `steps` Adam steps on <C> with
// adjoint gradients and then one forward pass that returns <C> and the top-k bitstrings at the
// final parameters (the paper's per-sub-QUBO optimise-then-sample loop of Section IV, with Adam
// in place of COBYLA). Jobs are admitted from a FIFO queue while a job slot and enough scratch
// memory (the streaming tier's per-instance state buffers) are free. Every tick runs one step of
// every admitted job in one batched launch (a plan placed in memory the server owns, so no
// allocation happens after creation); a job admitted while others are running joins at the next
// tick, and a finished job leaves at the end of its tick, so the batch changes tick by tick.
// Parameters, Adam moments, gradients and Q stay on the device in the job's slot for the
// job's whole life. The kernels are batch-invariant, so a job's results do not depend on what
// else shares its ticks.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <deque>
#include <vector>

#include "../../include/qaoa.h"
#include "qaoa_common.cuh"
#include "qaoa_host.h"

namespace {

constexpr int QSTRIDE = 1024;   // floats per job slot of the Q pool (n <= 30: n * n <= 900)
constexpr int PSTRIDE = 128;    // parameters per job slot (gamma[p], beta[p], p <= 64)
constexpr int RING = 3;         // ticks in flight

struct DevResult {
    double expect;
    uint64_t idx[16];
    double prob[16];
    float params[PSTRIDE];
};
struct AdamRow {
    int slot, p, step;
    float lr;
};
struct GatherRow {
    int inst, slot, p, pad;
};

__global__ void __launch_bounds__(PSTRIDE) k_adam_jobs(const AdamRow* __restrict__ rows,
                                                      float* __restrict__ ppool,
                                                      const double* __restrict__ gpool,
                                                      float* __restrict__ mpool, float* __restrict__ vpool) {
    const AdamRow r = rows[blockIdx.x];
    const int i = threadIdx.x;
    if (i >= 2 * r.p) return;
    const size_t o = (size_t)r.slot * PSTRIDE + i;
    qaoa::adam_update(ppool[o], mpool[o], vpool[o], gpool[o], r.step, r.lr, 0.9f, 0.999f, 1e-8f, 1);
}

__global__ void __launch_bounds__(PSTRIDE) k_gather_results(const GatherRow* __restrict__ rows, int K,
                                                           const double* __restrict__ expect,
                                                           const uint64_t* __restrict__ tidx,
                                                           const double* __restrict__ tprob,
                                                           const float* __restrict__ ppool,
                                                           DevResult* __restrict__ out) {
    const GatherRow r = rows[blockIdx.x];
    DevResult& o = out[blockIdx.x];
    const int t = threadIdx.x;
    if (t == 0) o.expect = expect[r.inst];
    if (t < 16) {
        o.idx[t] = t < K ? tidx[(size_t)r.inst * K + t] : 0;
        o.prob[t] = t < K ? tprob[(size_t)r.inst * K + t] : -1.0;
    }
    o.params[t] = t < 2 * r.p ? ppool[(size_t)r.slot * PSTRIDE + t] : 0.0f;
}

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Job {
    int64_t id;
    int n, p, steps, done;
    float lr;
    int slot;
    size_t foot;
    int state;  // 1 training, 2 final forward pending
    double t_submit;
    std::vector<float> Q, par;
};

struct TickRec {
    cudaEvent_t ev = nullptr;          // end of the tick's device work
    cudaEvent_t ev0 = nullptr;         // start (timing)
    char* host = nullptr;              // pinned: header staging | adam rows | gather rows | uploads | results
    std::vector<Job*> finishing;       // jobs whose results this tick copies back (results order)
    bool busy = false;
};

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct qaoa_server {
    qaoa_ctx* ctx = nullptr;
    int device = 0, max_jobs = 0, K = 0;
    size_t scratch_cap = 0, hdr_bound = 0, plan_bytes = 0;
    char* dev = nullptr;
    float *qpool = nullptr, *ppool = nullptr, *mpool = nullptr, *vpool = nullptr;
    double* gpool = nullptr;
    double* t_expect = nullptr;
    uint64_t* t_tidx = nullptr;
    double* t_tprob = nullptr;
    AdamRow* d_adam = nullptr;
    GatherRow* d_gather = nullptr;
    DevResult* d_res = nullptr;
    char* plan_mem = nullptr;
    size_t off_adam = 0, off_gather = 0, off_up = 0, off_res = 0, host_bytes = 0;
    TickRec ring[RING];
    long tick_no = 0;
    std::deque<Job*> queue;
    std::vector<Job*> active;
    std::vector<int> free_slots;
    size_t used = 0;
    std::vector<qaoa_job_result> done;
    int64_t next_id = 1;
    double bytes_total = 0.0;   // algorithmic DRAM bytes of every launched tick
    double gpu_ms_total = 0.0;  // device time of the harvested ticks
    long long launches = 0;     // kernel launches enqueued
    int fail_next = 0;          // admissions still to fail (qaoa_server_fail_admissions)
    long long admit_failures = 0;
};

namespace {

void harvest(qaoa_server* s, TickRec& R) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, R.ev0, R.ev) == cudaSuccess) s->gpu_ms_total += ms;
    const DevResult* res = reinterpret_cast<const DevResult*>(R.host + s->off_res);
    const double t = now_s();
    for (size_t r = 0; r < R.finishing.size(); ++r) {
        Job* j = R.finishing[r];
        qaoa_job_result o{};
        o.job_id = j->id;
        o.n = j->n;
        o.p = j->p;
        o.steps = j->steps;
        o.k = s->K;
        o.expect = res[r].expect;
        for (int i = 0; i < 16; ++i) {
            o.topk_idx[i] = res[r].idx[i];
            o.topk_prob[i] = res[r].prob[i];
        }
        for (int i = 0; i < PSTRIDE; ++i) o.params[i] = res[r].params[i];
        o.t_submit = j->t_submit;
        o.t_done = t;
        s->done.push_back(o);
        delete j;
    }
    R.finishing.clear();
    R.busy = false;
}

qaoa_status cuda_err(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof(buf), "server %s: %s", what, cudaGetErrorString(e));
    return qaoa::set_error(QAOA_E_CUDA, buf);
}

#define SCK(call, what)                                        \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_err(e_, what);      \
    } while (0)

}  // namespace

extern "C" double qaoa_server_clock(void) { return now_s(); }

extern "C" qaoa_status qaoa_server_create(qaoa_ctx* ctx, size_t scratch_bytes, int max_jobs, int k,
                                          qaoa_server** out) {
    if (!ctx || !out || max_jobs < 1 || max_jobs > 65536 || k < 0 || k > 16)
        return qaoa::set_error(QAOA_E_INVALID, "server_create: bad arguments");
    *out = nullptr;
    int device = 0;
    SCK(cudaGetDevice(&device), "cudaGetDevice");
    qaoa_server* s = new qaoa_server();
    s->ctx = ctx;
    s->device = device;
    s->max_jobs = max_jobs;
    s->K = k;
    s->scratch_cap = scratch_bytes;
    s->hdr_bound = qaoa::plan_header_bound(max_jobs);
    s->plan_bytes = s->hdr_bound + scratch_bytes;
    const size_t J = (size_t)max_jobs, kk = (size_t)std::max(k, 1);
    size_t o = 0;
    const size_t o_q = o;      o = al(o + J * QSTRIDE * sizeof(float));
    const size_t o_p = o;      o = al(o + J * PSTRIDE * sizeof(float));
    const size_t o_m = o;      o = al(o + J * PSTRIDE * sizeof(float));
    const size_t o_v = o;      o = al(o + J * PSTRIDE * sizeof(float));
    const size_t o_g = o;      o = al(o + J * PSTRIDE * sizeof(double));
    const size_t o_e = o;      o = al(o + J * sizeof(double));
    const size_t o_ti = o;     o = al(o + J * kk * sizeof(uint64_t));
    const size_t o_tp = o;     o = al(o + J * kk * sizeof(double));
    const size_t o_a = o;      o = al(o + J * sizeof(AdamRow));
    const size_t o_gr = o;     o = al(o + J * sizeof(GatherRow));
    const size_t o_r = o;      o = al(o + J * sizeof(DevResult));
    const size_t o_plan = o;   o = al(o + s->plan_bytes);
    cudaError_t e = cudaMalloc(&s->dev, o);
    if (e != cudaSuccess) {
        delete s;
        return qaoa::set_error(QAOA_E_NOMEM, "server_create: device memory for the job pools and scratch");
    }
    s->qpool = reinterpret_cast<float*>(s->dev + o_q);
    s->ppool = reinterpret_cast<float*>(s->dev + o_p);
    s->mpool = reinterpret_cast<float*>(s->dev + o_m);
    s->vpool = reinterpret_cast<float*>(s->dev + o_v);
    s->gpool = reinterpret_cast<double*>(s->dev + o_g);
    s->t_expect = reinterpret_cast<double*>(s->dev + o_e);
    s->t_tidx = reinterpret_cast<uint64_t*>(s->dev + o_ti);
    s->t_tprob = reinterpret_cast<double*>(s->dev + o_tp);
    s->d_adam = reinterpret_cast<AdamRow*>(s->dev + o_a);
    s->d_gather = reinterpret_cast<GatherRow*>(s->dev + o_gr);
    s->d_res = reinterpret_cast<DevResult*>(s->dev + o_r);
    s->plan_mem = s->dev + o_plan;
    size_t h = s->hdr_bound;
    s->off_adam = h;   h = al(h + J * sizeof(AdamRow));
    s->off_gather = h; h = al(h + J * sizeof(GatherRow));
    s->off_up = h;     h = al(h + J * (QSTRIDE + PSTRIDE) * sizeof(float));
    s->off_res = h;    h = al(h + J * sizeof(DevResult));
    s->host_bytes = h;
    for (auto& R : s->ring) {
        if (cudaMallocHost(&R.host, s->host_bytes) != cudaSuccess ||
            cudaEventCreate(&R.ev) != cudaSuccess || cudaEventCreate(&R.ev0) != cudaSuccess) {
            qaoa_server_destroy(s);
            return qaoa::set_error(QAOA_E_NOMEM, "server_create: pinned staging");
        }
    }
    for (int i = max_jobs - 1; i >= 0; --i) s->free_slots.push_back(i);
    *out = s;
    return QAOA_OK;
}

extern "C" void qaoa_server_destroy(qaoa_server* s) {
    if (!s) return;
    cudaSetDevice(s->device);
    cudaDeviceSynchronize();
    for (auto& R : s->ring) {
        for (Job* j : R.finishing) delete j;
        if (R.host) cudaFreeHost(R.host);
        if (R.ev) cudaEventDestroy(R.ev);
        if (R.ev0) cudaEventDestroy(R.ev0);
    }
    for (Job* j : s->queue) delete j;
    for (Job* j : s->active) delete j;
    if (s->dev) cudaFree(s->dev);
    delete s;
}

extern "C" size_t qaoa_server_job_bytes(qaoa_server* s, int n, int p) {
    if (!s || n < 1 || n > 30 || p < 1 || p > 64) return 0;
    return std::max(qaoa::plan_inst_scratch_bytes(s->ctx, n, p, 0, true),
                    qaoa::plan_inst_scratch_bytes(s->ctx, n, p, s->K, false));
}

extern "C" qaoa_status qaoa_server_submit(qaoa_server* s, int n, int p, const float* Q, const float* params,
                                          int steps, float lr, int64_t* job_id) {
    if (!s || n < 1 || n > 30 || p < 1 || p > 64 || !Q || !params || steps < 0 || !(lr > 0.0f) ||
        (uint64_t)s->K > (1ull << n))
        return qaoa::set_error(QAOA_E_INVALID, "server_submit: bad arguments");
    Job* j = new Job();
    j->id = s->next_id++;
    j->n = n;
    j->p = p;
    j->steps = steps;
    j->done = 0;
    j->lr = lr;
    j->slot = -1;
    j->foot = al(qaoa_server_job_bytes(s, n, p));
    if (j->foot > s->scratch_cap) {
        delete j;
        return qaoa::set_error(QAOA_E_NOMEM, "server_submit: the job needs more scratch than the server has");
    }
    j->state = steps > 0 ? 1 : 2;
    j->t_submit = now_s();
    j->Q.assign(Q, Q + (size_t)n * n);
    j->par.assign(params, params + 2 * p);
    s->queue.push_back(j);
    if (job_id) *job_id = j->id;
    return QAOA_OK;
}

extern "C" qaoa_status qaoa_server_tick(qaoa_server* s, qaoa_stream_t stream, int* active_out, int* queued_out) {
    if (!s) return qaoa::set_error(QAOA_E_INVALID, "server_tick: NULL server");
    cudaStream_t st = (cudaStream_t)stream;
    SCK(cudaSetDevice(s->device), "cudaSetDevice");
    TickRec& R = s->ring[s->tick_no % RING];
    if (R.busy) {                                   // back-pressure: at most RING ticks in flight
        SCK(cudaEventSynchronize(R.ev), "cudaEventSynchronize");
        harvest(s, R);
    }
    SCK(cudaEventRecord(R.ev0, st), "cudaEventRecord");
    // ---- admission: FIFO while a slot and the job's scratch are free ----
    float* up = reinterpret_cast<float*>(R.host + s->off_up);
    size_t upn = 0;
    while (!s->queue.empty() && !s->free_slots.empty() && s->used + s->queue.front()->foot <= s->scratch_cap) {
        if (s->fail_next > 0) {
            // the job's scratch could not be had: it keeps its place at the head of the queue
            // (FIFO, nobody overtakes it) and admission resumes at the next tick
            --s->fail_next;
            ++s->admit_failures;
            break;
        }
        Job* j = s->queue.front();
        s->queue.pop_front();
        j->slot = s->free_slots.back();
        s->free_slots.pop_back();
        s->used += j->foot;
        float* uq = up + upn;
        std::memcpy(uq, j->Q.data(), j->Q.size() * sizeof(float));
        std::memcpy(uq + j->Q.size(), j->par.data(), j->par.size() * sizeof(float));
        SCK(cudaMemcpyAsync(s->qpool + (size_t)j->slot * QSTRIDE, uq, j->Q.size() * sizeof(float),
                            cudaMemcpyHostToDevice, st), "upload Q");
        SCK(cudaMemcpyAsync(s->ppool + (size_t)j->slot * PSTRIDE, uq + j->Q.size(), j->par.size() * sizeof(float),
                            cudaMemcpyHostToDevice, st), "upload parameters");
        SCK(cudaMemsetAsync(s->mpool + (size_t)j->slot * PSTRIDE, 0, PSTRIDE * sizeof(float), st), "zero m");
        SCK(cudaMemsetAsync(s->vpool + (size_t)j->slot * PSTRIDE, 0, PSTRIDE * sizeof(float), st), "zero v");
        upn += j->Q.size() + j->par.size();
        j->Q.clear();
        j->Q.shrink_to_fit();
        s->active.push_back(j);
    }
    if (active_out) *active_out = (int)s->active.size();
    if (queued_out) *queued_out = (int)s->queue.size();
    if (s->active.empty()) {
        SCK(cudaEventRecord(R.ev, st), "cudaEventRecord");
        R.busy = true;
        ++s->tick_no;
        return QAOA_OK;
    }
    // ---- one batched launch: a gradient step for training jobs, the final forward pass with
    // top-k for jobs that finished training ----
    std::vector<qaoa_inst> desc;
    desc.reserve(s->active.size());
    for (Job* j : s->active) {
        qaoa_inst d{};
        d.n = j->n;
        d.p = j->p;
        d.k = j->state == 2 ? s->K : 0;
        d.flags = j->state == 1 ? QAOA_INST_GRAD : 0;
        d.q_off = (int64_t)j->slot * QSTRIDE;
        d.par_off = (int64_t)j->slot * PSTRIDE;
        d.psi_off = -1;
        d.e_off = -1;
        desc.push_back(d);
    }
    qaoa_batch_io io{};
    io.q = s->qpool;
    io.params = s->ppool;
    io.expect = s->t_expect;
    io.topk_idx = s->t_tidx;
    io.topk_prob = s->t_tprob;
    io.k_stride = std::max(s->K, 1);
    io.grad = s->gpool;
    qaoa_plan* plan = nullptr;
    qaoa_status q = qaoa::plan_create_placed(s->ctx, desc.data(), (int)desc.size(), &io, s->plan_mem,
                                             s->plan_bytes, st, R.host, s->hdr_bound, &plan);
    if (q != QAOA_OK) return q;
    q = qaoa_plan_launch(plan, st);
    {
        s->launches += qaoa_plan_kernel_count(plan);
        std::vector<double> kb(qaoa_plan_kernel_count(plan) + 8);
        const int nk = qaoa_plan_kernel_bytes(plan, kb.data(), (int)kb.size());
        for (int i = 0; i < nk; ++i) s->bytes_total += kb[i];
    }
    qaoa_plan_destroy(plan);   // placed plan: host bookkeeping only, the launch is already queued
    if (q != QAOA_OK) return q;
    // ---- Adam on the training jobs, results of the finishing ones ----
    AdamRow* ar = reinterpret_cast<AdamRow*>(R.host + s->off_adam);
    GatherRow* gr = reinterpret_cast<GatherRow*>(R.host + s->off_gather);
    int na = 0, ng = 0;
    std::vector<Job*> keep;
    keep.reserve(s->active.size());
    for (size_t i = 0; i < s->active.size(); ++i) {
        Job* j = s->active[i];
        if (j->state == 1) {
            ar[na++] = AdamRow{j->slot, j->p, j->done + 1, j->lr};
            if (++j->done >= j->steps) j->state = 2;
            keep.push_back(j);
        } else {
            gr[ng++] = GatherRow{(int)i, j->slot, j->p, 0};
            R.finishing.push_back(j);
            s->free_slots.push_back(j->slot);   // later reuse is stream-ordered after this tick
            s->used -= j->foot;
        }
    }
    if (na) {
        SCK(cudaMemcpyAsync(s->d_adam, ar, na * sizeof(AdamRow), cudaMemcpyHostToDevice, st), "upload adam rows");
        k_adam_jobs<<<na, PSTRIDE, 0, st>>>(s->d_adam, s->ppool, s->gpool, s->mpool, s->vpool);
        SCK(cudaGetLastError(), "k_adam_jobs");
        ++s->launches;
    }
    if (ng) {
        SCK(cudaMemcpyAsync(s->d_gather, gr, ng * sizeof(GatherRow), cudaMemcpyHostToDevice, st), "upload gather rows");
        k_gather_results<<<ng, PSTRIDE, 0, st>>>(s->d_gather, s->K, s->t_expect, s->t_tidx, s->t_tprob,
                                                 s->ppool, s->d_res);
        SCK(cudaGetLastError(), "k_gather_results");
        ++s->launches;
        SCK(cudaMemcpyAsync(R.host + s->off_res, s->d_res, ng * sizeof(DevResult), cudaMemcpyDeviceToHost, st),
            "copy results");
    }
    s->active.swap(keep);
    SCK(cudaEventRecord(R.ev, st), "cudaEventRecord");
    R.busy = true;
    ++s->tick_no;
    return QAOA_OK;
}

extern "C" qaoa_status qaoa_server_cancel(qaoa_server* s, int64_t job_id) {
    if (!s) return qaoa::set_error(QAOA_E_INVALID, "server_cancel: NULL server");
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        if ((*it)->id != job_id) continue;
        delete *it;
        s->queue.erase(it);
        return QAOA_OK;
    }
    for (auto it = s->active.begin(); it != s->active.end(); ++it) {
        Job* j = *it;
        if (j->id != job_id) continue;
        // an admitted job leaves between ticks: the ticks already enqueued still read its slot,
        // and a job admitted into the slot later uploads its inputs behind them on the stream
        s->free_slots.push_back(j->slot);
        s->used -= j->foot;
        delete j;
        s->active.erase(it);
        return QAOA_OK;
    }
    return qaoa::set_error(QAOA_E_INVALID, "server_cancel: the job is not queued or running (unknown, or its "
                           "final pass is already enqueued)");
}

extern "C" qaoa_status qaoa_server_fail_admissions(qaoa_server* s, int count, long long* failures) {
    if (!s || count < 0) return qaoa::set_error(QAOA_E_INVALID, "server_fail_admissions: bad arguments");
    s->fail_next = count;
    if (failures) *failures = s->admit_failures;
    return QAOA_OK;
}

extern "C" int qaoa_server_poll(qaoa_server* s, int wait, qaoa_job_result* out, int max) {
    if (!s) return -1;
    cudaSetDevice(s->device);
    for (auto& R : s->ring) {
        if (!R.busy) continue;
        if (wait) cudaEventSynchronize(R.ev);
        else if (cudaEventQuery(R.ev) != cudaSuccess) continue;
        harvest(s, R);
    }
    const int n = std::min<int>(max, (int)s->done.size());
    if (out && n > 0) {
        std::memcpy(out, s->done.data(), n * sizeof(qaoa_job_result));
        s->done.erase(s->done.begin(), s->done.begin() + n);
    }
    return n;
}

extern "C" qaoa_status qaoa_server_stats(qaoa_server* s, int* queued, int* active, size_t* scratch_used,
                                         double* bytes_total, double* gpu_ms_total, long long* launches) {
    if (!s) return qaoa::set_error(QAOA_E_INVALID, "server_stats: NULL server");
    if (queued) *queued = (int)s->queue.size();
    if (active) *active = (int)s->active.size();
    if (scratch_used) *scratch_used = s->used;
    if (bytes_total) *bytes_total = s->bytes_total;
    if (gpu_ms_total) *gpu_ms_total = s->gpu_ms_total;
    if (launches) *launches = s->launches;
    return QAOA_OK;
}
