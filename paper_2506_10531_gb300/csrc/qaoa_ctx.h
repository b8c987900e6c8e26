// qaoa_ctx.h -- the library context (internal): device, workspace, tier overrides and the
// autotuner's table of measured best configurations.
#pragma once
#include <stddef.h>

#include "../../include/qaoa.h"
#include "qaoa_kernels.h"

// One autotuned choice for complex64 batches of (n, p): the kernel tier and, for the cluster
// tier, the local qubits per CTA; ms is the measured batch time it won with.
struct qaoa_tuned {
    int tier = 0;  // 0: not tuned
    int L = 0;
    double ms = 0.0;
    int count = 0, k = 0;
};

struct qaoa_ctx {
    int device = 0;
    int nsm = 0;
    void* ws = nullptr;       // workspace (device)
    size_t ws_bytes = 0;
    int* queue = nullptr;     // work counters of the single-call launches (device)
    int tier[32] = {0};       // QAOA_TIER_* per n for complex64 plans (0: automatic)
    int cluster_L[32] = {0};  // local qubits per CTA of the cluster tier by n (0: default 14)
    qaoa_tuned tuned[32][65]; // autotuner table by (n, p)
    int cs_ok[32] = {0};      // cluster-streaming tier: 0 unknown, 1 usable, -1 not on this device
};

namespace qaoa {
// Tier of a complex64 instance of (n, p) without gradient above the resident range: an explicit
// qaoa_set_tier wins, then the autotuner's entry, then the default: the cluster-streaming tier for
// n = 15..17, the streaming tier above.
inline int eff_tier(const qaoa_ctx* c, int n, int p) {
    if (c->tier[n]) return c->tier[n];
    if (p >= 1 && p <= 64 && c->tuned[n][p].tier) return c->tuned[n][p].tier;
    return (n >= 15 && n <= 17) ? QAOA_TIER_CSTREAM : QAOA_TIER_STREAM;
}
// The cluster-streaming tier can run n-qubit instances on the context's device (tensor-map
// encoder found, a cluster of its shape fits); cached per n.
bool cstream_usable(qaoa_ctx* c, int n);
// Widest forward register window of the resident tier (complex64) for (n, p): qaoa_set_tier's
// param with QAOA_TIER_RESIDENT, else the autotuner's choice, else 4 qubits for n <= 12 (twice
// the threads per instance: measured on GB300 6-17% faster for batches of n = 8..12) and 5 above
// (n = 14: 12% slower with 4).
inline int eff_resident_rmax(const qaoa_ctx* c, int n, int p) {
    if (c->tier[n] == QAOA_TIER_RESIDENT && c->cluster_L[n]) return c->cluster_L[n];
    if (p >= 1 && p <= 64 && c->tuned[n][p].tier == QAOA_TIER_RESIDENT && c->tuned[n][p].L) return c->tuned[n][p].L;
    return n <= 12 ? 4 : RES_RMAX;
}
// Variant of the HBM-streaming tier's forward passes: 0 TMA passes with two CTAs per SM, 1 TMA
// passes with one CTA per SM, 2 the per-thread cp.async passes (qaoa_set_tier's param, else the
// autotuner's, else 0).
inline int eff_stream_variant(const qaoa_ctx* c, int n, int p) {
    if (c->tier[n] == QAOA_TIER_STREAM) return c->cluster_L[n];
    if (p >= 1 && p <= 64 && c->tuned[n][p].tier == QAOA_TIER_STREAM) return c->tuned[n][p].L;
    return 0;
}
inline int eff_cluster_L(const qaoa_ctx* c, int n, int p) {
    if (c->tier[n] == QAOA_TIER_CLUSTER && c->cluster_L[n]) return c->cluster_L[n];
    if (p >= 1 && p <= 64 && c->tuned[n][p].tier == QAOA_TIER_CLUSTER && c->tuned[n][p].L) return c->tuned[n][p].L;
    return 13;
}
}  // namespace qaoa
