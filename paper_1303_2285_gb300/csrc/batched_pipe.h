// Host side of the batched plan's stage form (batched_pipe.cu): every member
// runs through the stages of the single-matrix combination path, each stage
// one launch over all members (internal).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

#include "../../include/cov.h"
#include "cov_internal.h"

namespace cov {

// Members grouped by a template parameter of a stage's kernel: the shared-
// memory pitch of the product tiles, or the column-lag register count of the
// fringe-row tasks; the last two stages: every member (key 0 the reductions,
// key 1 the walk).
struct PipeClass {
  int key;                       // PITCH (products), QMAXF (fringe rows), 0 / 1 (last stages)
  std::vector<int> members;      // member indices, in launch order (products: per chunk)
  std::vector<long long> first;  // products: task range [a, b) of each chunk; otherwise a
                                 // prefix over the members (members + 1 entries): fringe-row
                                 // CTAs, reduction tasks or walk segments
  long long total = 0;           // chunks, or the prefix's last entry
  size_t counter = 0;            // products: workspace offset of the launch's chunk counter
  size_t smem = 0;               // dynamic shared memory of the launch
  size_t off_members = 0, off_first = 0;  // workspace offsets of the two arrays
};

struct PipePlan {
  int elem = 8;                  // bytes of one complex element (8: COV_C64, 16: COV_C128)
  // per member: the single-matrix plan, its pointer fields (status and the
  // partial-sum arrays) holding offsets into the workspace
  std::vector<RecParams> params;
  mutable std::vector<RecParams> resolved;  // params with the last upload's addresses
  std::vector<PipeClass> products, fringe, finish;
  size_t off_params = 0, total = 0;
};

// True if every member fits the stage form (the combination path's shape
// rule, 8-byte aligned A and R).
bool pipe_members_ok(const cov_desc *descs, int count);

// Plans every member (plan_recurrence, no tuning cache), groups the members,
// cuts the product tasks into chunks for `sms` SMs and lays out, from
// workspace offset `off`, the tables and each member's partial-sum arrays;
// pp.total = the end of the layout.
void pipe_plan_build(PipePlan &pp, const cov_desc *descs, int count, int elem, int mean,
                     size_t off, int sms);

// Copies the tables into the workspace, the member plans with their
// addresses in this workspace (stream-ordered; the plan must stay alive until
// the copies have run). The tables are valid for this workspace only.
cudaError_t pipe_upload(const PipePlan &pp, char *ws, cudaStream_t s);

// The launches: products, fringe rows, reductions, walk.
cudaError_t pipe_launch(const PipePlan &pp, char *ws, int sms, cudaStream_t s);

}  // namespace cov
