// Build plan: every stage of the Hamiltonian build as one grouped launch over
// all target-group pairs, target groups and L2 sets of one or many staged
// Hamiltonians (k_plan.cu).
#pragma once

#include <vector>

#include "hb_api_internal.cuh"

namespace hb {
struct Plan;
}

// Plan over n contexts (same orbital space: equal n_words, n_to and label
// count) writing into outs[i].  Prepares the tensor-core operands when
// precision is HB_MIXED.  Returns HB_OK or an error with *err set.
int plan_create(hb_ctx *const *ctxs, int n, const hb_blocks *outs, int precision, hb::Plan **out, std::string *err,
                cudaStream_t s, int shard_r = 0, int shard_n = 1);
// Phase of the next plan_run of a sharded plan: 1 the contraction only, 2 the
// rest, 0 everything; and whether a plan is the shard (precision, r, n).
void plan_set_phase(hb::Plan *p, int phase);
bool plan_is_shard(const hb::Plan *p, int precision, int r, int n);
// Point the plan's tasks at new output blocks (re-uploads the task tables).
int plan_set_outputs(hb::Plan *p, const hb_blocks *outs, std::string *err, cudaStream_t s);
bool plan_outputs_equal(const hb::Plan *p, const hb_blocks *outs);
int plan_precision(const hb::Plan *p);
// Issue every stage on stream s.  timing: record the stage events (as graph
// event nodes when capture is set).  *launches: kernels launched.
int plan_run(hb::Plan *p, cudaStream_t s, bool timing, bool capture, int *launches, std::string *err);
// After the stream has finished a timed run: per-stage times and counters.
void plan_stats(hb::Plan *p, hb_stats *st);
// Time the result-identical launch-shape candidates of every tunable stage
// (split tile arrangement, class-4 state tile and threads, gamma warp or block
// per key) on this plan's own tasks, keep the fastest, re-upload the tables.
int plan_autotune(hb::Plan *p, cudaStream_t s, std::string *err);
bool plan_tuned(const hb::Plan *p);
// The launch shapes in use, as text.
std::string plan_report(const hb::Plan *p);
// Bounded-wait status word of the tensor-core kernel (0: fine).
int plan_error_word(hb::Plan *p, int *word);
void plan_destroy(hb::Plan *p);
