// qaoa_tune.cu -- autotuner and tuning table of libqaoa.
//
// For complex64 batches of `count` instances of (n, p) with top-k length k the tuner times every
// kernel configuration that can run them on synthetic inputs, with CUDA events around whole plan
// launches (best of several), and stores the fastest in the context. For 15 <= n <= 30: the
// HBM-streaming tier's three forward-pass variants (TMA passes with two CTAs per SM or one, the
// per-thread cp.async passes); for 15 <= n <= 18 also the DSMEM cluster tier with 13 or 14 local
// qubits per CTA (2^(n-L) CTAs per cluster, at most 16); for 15 <= n <= 17 the cluster-streaming
// tier; for 6 <= n <= 14 the resident tier with forward register windows of 5 qubits or (n <= 13)
// 4 qubits (blocks of 2^(n-5) or 2^(n-4) threads). Plans created afterwards use the stored choice unless qaoa_set_tier
// overrides it. The table is saved and loaded as a small JSON document, so a sweep done once
// per machine can be reused (the offline sweep / online cache split).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/qaoa.h"
#include "qaoa_cstream.h"
#include "qaoa_ctx.h"
#include "qaoa_host.h"

namespace {

qaoa_status cuda_err(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof(buf), "autotune %s: %s", what, cudaGetErrorString(e));
    return qaoa::set_error(QAOA_E_CUDA, buf);
}

#define TCK(call, what)                                        \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_err(e_, what);      \
    } while (0)

// Deterministic synthetic inputs: Q entries uniform in [-1, 1] from a 64-bit LCG, symmetric.
void synth_q(int n, int count, std::vector<float>& q) {
    q.assign((size_t)count * n * n, 0.0f);
    uint64_t x = 0x2545F4914F6CDD1Dull;
    for (int b = 0; b < count; ++b)
        for (int i = 0; i < n; ++i)
            for (int j = i; j < n; ++j) {
                x = x * 6364136223846793005ull + 1442695040888963407ull;
                const float v = (float)((double)(x >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
                q[(size_t)b * n * n + i * n + j] = v;
                q[(size_t)b * n * n + j * n + i] = v;
            }
}

struct Candidate {
    int tier, L;
};

}  // namespace

extern "C" qaoa_status qaoa_autotune(qaoa_ctx* c, int n, int p, int k, int count, qaoa_stream_t stream,
                                     double* best_ms) {
    if (!c || n < 1 || n > 30 || p < 1 || p > 64 || k < 0 || k > 16 || count < 1 || (uint64_t)k > (1ull << n))
        return qaoa::set_error(QAOA_E_INVALID, "autotune: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    TCK(cudaSetDevice(c->device), "cudaSetDevice");
    std::vector<Candidate> cand;
    if (n >= 15) {
        if (n <= qaoa::CS_NMAX && qaoa::cstream_usable(c, n)) cand.push_back({QAOA_TIER_CSTREAM, 0});
        if (n <= 18)
            for (int L = 14; L >= 13; --L)
                if (n - L >= 1 && n - L <= 4) cand.push_back({QAOA_TIER_CLUSTER, L});
        for (int v = 0; v <= 2; ++v) cand.push_back({QAOA_TIER_STREAM, v});
    } else if (n >= 6) {
        cand.push_back({QAOA_TIER_RESIDENT, 5});
        if (n <= 13) cand.push_back({QAOA_TIER_RESIDENT, 4});
    } else {
        cand.push_back({0, 0});   // one configuration: time it, store nothing
    }
    // inputs
    std::vector<float> qh;
    synth_q(n, count, qh);
    std::vector<float> ph(2 * p);
    for (int l = 0; l < p; ++l) {
        ph[l] = 0.2f + 0.1f * l;
        ph[p + l] = 0.6f - 0.05f * l;
    }
    float *qd = nullptr, *pd = nullptr;
    double *ex = nullptr, *tp = nullptr;
    uint64_t* ti = nullptr;
    const size_t kk = (size_t)std::max(k, 1);
    TCK(cudaMalloc(&qd, qh.size() * sizeof(float)), "cudaMalloc");
    cudaMalloc(&pd, ph.size() * sizeof(float));
    cudaMalloc(&ex, (size_t)count * sizeof(double));
    cudaMalloc(&ti, (size_t)count * kk * sizeof(uint64_t));
    cudaMalloc(&tp, (size_t)count * kk * sizeof(double));
    auto release = [&]() {
        cudaFree(qd);
        cudaFree(pd);
        cudaFree(ex);
        cudaFree(ti);
        cudaFree(tp);
    };
    if (!pd || !ex || !ti || !tp) {
        release();
        return qaoa::set_error(QAOA_E_NOMEM, "autotune: input buffers");
    }
    cudaMemcpy(qd, qh.data(), qh.size() * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(pd, ph.data(), ph.size() * sizeof(float), cudaMemcpyHostToDevice);
    std::vector<qaoa_inst> desc(count);
    for (int i = 0; i < count; ++i) desc[i] = qaoa_inst{n, p, k, 0, (int64_t)i * n * n, 0, -1, -1};
    qaoa_batch_io io{};
    io.q = qd;
    io.params = pd;
    io.expect = ex;
    io.topk_idx = k ? ti : nullptr;
    io.topk_prob = k ? tp : nullptr;
    io.k_stride = (int)kk;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int saved_tier = c->tier[n], saved_L = c->cluster_L[n];
    double best = -1.0;
    Candidate win{0, 0};
    qaoa_status status = QAOA_OK;
    for (const Candidate& cd : cand) {
        c->tier[n] = cd.tier;
        c->cluster_L[n] = cd.L;
        qaoa_plan* plan = nullptr;
        qaoa_status q = qaoa_plan_create(c, desc.data(), count, &io, 0, &plan);
        if (q == QAOA_E_UNSUPPORTED || q == QAOA_E_NOMEM) continue;   // configuration cannot run here
        if (q != QAOA_OK) { status = q; break; }
        double t = 1e30;
        for (int r = 0; r < 2 && q == QAOA_OK; ++r) q = qaoa_plan_launch(plan, stream);
        for (int r = 0; r < 5 && q == QAOA_OK; ++r) {
            cudaEventRecord(e0, st);
            q = qaoa_plan_launch(plan, stream);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            t = std::min(t, (double)ms);
        }
        qaoa_plan_destroy(plan);
        if (q != QAOA_OK) { status = q; break; }
        if (best < 0.0 || t < best) {
            best = t;
            win = cd;
        }
    }
    c->tier[n] = saved_tier;
    c->cluster_L[n] = saved_L;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    release();
    if (status != QAOA_OK) return status;
    if (best < 0.0) return qaoa::set_error(QAOA_E_UNSUPPORTED, "autotune: no configuration runs");
    if (win.tier) {
        qaoa_tuned& t = c->tuned[n][p];
        t.tier = win.tier;
        t.L = win.L;
        t.ms = best;
        t.count = count;
        t.k = k;
    }
    if (best_ms) *best_ms = best;
    return QAOA_OK;
}

extern "C" qaoa_status qaoa_tuning_get(qaoa_ctx* c, int n, int p, int* tier, int* param, double* ms) {
    if (!c || n < 1 || n > 30 || p < 1 || p > 64) return qaoa::set_error(QAOA_E_INVALID, "tuning_get: bad arguments");
    const qaoa_tuned& t = c->tuned[n][p];
    if (tier) *tier = t.tier;
    if (param) *param = t.L;
    if (ms) *ms = t.ms;
    return QAOA_OK;
}

extern "C" qaoa_status qaoa_tuning_save(qaoa_ctx* c, const char* path) {
    if (!c || !path) return qaoa::set_error(QAOA_E_INVALID, "tuning_save: bad arguments");
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, c->device);
    FILE* f = fopen(path, "w");
    if (!f) return qaoa::set_error(QAOA_E_INVALID, "tuning_save: cannot open the file");
    fprintf(f, "{\"format\": \"libqaoa-tuning-1\", \"device\": \"%s\", \"sms\": %d, \"entries\": [", prop.name,
            prop.multiProcessorCount);
    bool first = true;
    for (int n = 1; n <= 30; ++n)
        for (int p = 1; p <= 64; ++p) {
            const qaoa_tuned& t = c->tuned[n][p];
            if (!t.tier) continue;
            fprintf(f, "%s\n  {\"n\": %d, \"p\": %d, \"tier\": %d, \"L\": %d, \"ms\": %.6f, \"count\": %d, \"k\": %d}",
                    first ? "" : ",", n, p, t.tier, t.L, t.ms, t.count, t.k);
            first = false;
        }
    fprintf(f, "\n]}\n");
    const bool ok = fclose(f) == 0;
    return ok ? QAOA_OK : qaoa::set_error(QAOA_E_INVALID, "tuning_save: write failed");
}

extern "C" qaoa_status qaoa_tuning_load(qaoa_ctx* c, const char* path) {
    if (!c || !path) return qaoa::set_error(QAOA_E_INVALID, "tuning_load: bad arguments");
    FILE* f = fopen(path, "r");
    if (!f) return qaoa::set_error(QAOA_E_INVALID, "tuning_load: cannot open the file");
    std::string text;
    char buf[4096];
    size_t r;
    while ((r = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, r);
    fclose(f);
    if (text.find("\"libqaoa-tuning-1\"") == std::string::npos)
        return qaoa::set_error(QAOA_E_INVALID, "tuning_load: not a libqaoa tuning file");
    size_t pos = 0;
    while ((pos = text.find("{\"n\":", pos)) != std::string::npos) {
        int n = 0, p = 0, tier = 0, L = 0, cnt = 0, k = 0;
        double ms = 0.0;
        if (sscanf(text.c_str() + pos, "{\"n\": %d, \"p\": %d, \"tier\": %d, \"L\": %d, \"ms\": %lf, \"count\": %d, \"k\": %d}",
                   &n, &p, &tier, &L, &ms, &cnt, &k) == 7 &&
            n >= 1 && n <= 30 && p >= 1 && p <= 64 && (tier == QAOA_TIER_RESIDENT || n >= 15) &&
            ((tier == QAOA_TIER_STREAM && L >= 0 && L <= 2) || (tier == QAOA_TIER_CSTREAM && n <= qaoa::CS_NMAX) ||
             (tier == QAOA_TIER_RESIDENT && n <= 14 && ((L == 4 && n <= 13) || L == 5)) ||
             (tier == QAOA_TIER_CLUSTER && n <= 18 && n - L >= 1 && n - L <= 4 && L >= 10))) {
            qaoa_tuned& t = c->tuned[n][p];
            t.tier = tier;
            t.L = L;
            t.ms = ms;
            t.count = cnt;
            t.k = k;
        }
        ++pos;
    }
    return QAOA_OK;
}
