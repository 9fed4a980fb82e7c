// evr_persist.cuh -- the batch's persistent step (evr_persist.cu): one launch runs a
// whole step of a batch of streams from a work queue.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

#include "evr_internal.cuh"

namespace evr {

// Control words of the persistent step (device ints, zero between launches; the launch's
// last CTA to leave resets them): the next work item, the CTAs that have left, the
// abort flag, the step's status (a timeout; kept until the host clears it), then per
// stream its completed work items, one 128-byte line each (waiting CTAs poll them).
constexpr int kCtrlHead = 0, kCtrlLeft = 1, kCtrlAbort = 2, kCtrlStatus = 3;
constexpr int kCtrlCount = 32, kCtrlStride = 32;
inline size_t persist_ctrl_ints(int n_streams) {
  return (size_t)kCtrlCount + (size_t)kCtrlStride * n_streams;
}

// Rows of one prologue work item.
constexpr int kPersistProRows = 16;

// A work item (int4): x = stream, y = what (-2 its packet's push, -1 a band of
// kPersistProRows rows of its prologue, j >= 0 pass j), z = band or tile index, w = the
// stream's completed items the item waits for.
constexpr int kItemPush = -2, kItemPrologue = -1;

struct PersistArgs {
  const Planes* descs;
  int* curs;
  int* active;
  const int4* items;
  const int* totals;  // per stream: its work items in the step
  int* ctrl;
  int n_items;
  int n_streams;
  int R, iters;  // pass j runs min(R, iters - j R) iterations
  int timing;    // autotuner trials: passes only, each from the live buffer into the
                 // other one, every stream taken as active, no flip
  SolveConsts c;
  PrologueConsts pc;
  const uint16_t* x;
  const uint16_t* y;
  const long long* t;
  const int8_t* pol;
  const long long* offsets;
};

// Whether the persistent step is instantiated for this configuration's tile and storage.
bool persist_supported(const SolverCfg& cfg, int storage);
// CTAs of the launch: resident CTAs per SM x SMs (0 on error).
int persist_grid(const SolverCfg& cfg, int storage);
int launch_batch_persist(const SolverCfg& cfg, int storage, const PersistArgs& a, int grid,
                         cudaStream_t st);
// A captured launch's node takes new arguments (the next step's packets).
int persist_node_set(cudaGraphExec_t exec, cudaGraphNode_t node, const PersistArgs& a);

}  // namespace evr
