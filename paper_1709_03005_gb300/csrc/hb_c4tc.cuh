// Class 4 of the mixed build on the tensor cores (k_class4_tc.cu): per-context
// operand tables and term lists, and the grouped launches of a build.
#pragma once

#include <vector>

#include "hb_api_internal.cuh"
#include "hb_tasks.cuh"

namespace hb {

// Make the integral slices (or borrow the base context's), the CI slices of
// every group with 1..64 states and the term-list row pointers (this runs the
// class-4 classification once).  S: slices per operand.
int c4tc_prepare(hb_ctx *ctx, int S, cudaStream_t s);
// Whether group g of ctx has tensor-core class-4 operands.
bool c4tc_group_on(const hb_ctx *ctx, int g);
// The term-fill and kernel tasks of group g writing into Hlc, with their
// block / work-item counts.
void c4tc_tasks(const hb_ctx *ctx, int g, double *Hlc, C4FTask *fill, int64_t *fill_blocks, C4TTask *tc,
                int64_t *tc_items);
// The work items of group g (task index ti of the launch) appended to *items.
void c4tc_items(const hb_ctx *ctx, int g, int ti, std::vector<C4Item> *items);
int g_c4fill(const Grouped<C4FTask> &g, cudaStream_t s);
// S: slices (the same for every task of the launch); err: bounded-wait status word
int g_c4tc(const Grouped<C4TTask> &g, const C4Item *items, int n_items, int S, int *err, cudaStream_t s);
void release_c4tc(hb_ctx *ctx);

}  // namespace hb
