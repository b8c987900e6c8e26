// qaoa_ctx.h -- the library context (internal): device, workspace, tier overrides and the
// autotuner's table of measured best configurations.
#pragma once
#include <stddef.h>

#include "../../include/qaoa.h"

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
};

namespace qaoa {
// Tier of a complex64 instance of (n, p) without gradient in the 15..18 cluster range: an
// explicit qaoa_set_tier wins, then the autotuner's entry, then the default measured on GB300
// for batches of a few hundred instances at p = 3: the cluster tier with 13 local qubits for
// n = 15, the streaming tier for n = 16..18 (faster by 7%, 34% and 50%).
inline int eff_tier(const qaoa_ctx* c, int n, int p) {
    if (c->tier[n]) return c->tier[n];
    if (p >= 1 && p <= 64 && c->tuned[n][p].tier) return c->tuned[n][p].tier;
    return n == 15 ? QAOA_TIER_CLUSTER : QAOA_TIER_STREAM;
}
inline int eff_cluster_L(const qaoa_ctx* c, int n, int p) {
    if (c->tier[n] == QAOA_TIER_CLUSTER && c->cluster_L[n]) return c->cluster_L[n];
    if (p >= 1 && p <= 64 && c->tuned[n][p].tier == QAOA_TIER_CLUSTER && c->tuned[n][p].L) return c->tuned[n][p].L;
    return 13;
}
}  // namespace qaoa
