// Handles of the C-ABI (private to the library's translation units) and the
// host-side helpers that more than one of them uses.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/mr_lbm.h"
#include "mr_internal.cuh"

// One time step captured as a CUDA graph per mesh parity (the two meshes
// alternate), replayed by the step calls; the event-record nodes of a
// profiled kernel group are pointed at fresh events before each replay.
struct StepGraph {
  cudaGraphExec_t exec = nullptr;
  int prof = -1;
  long long launches = 0;
  std::vector<cudaGraphNode_t> ev_nodes;
  cudaGraph_t graph = nullptr;
};

// What queues time steps: a stream, the parity of the current mesh, the
// captured graphs, launch counting and the optional event timing of one
// kernel group.  A solver and a batch of solvers are both executors.
struct Exec {
  cudaStream_t st = nullptr;
  int nsm = 152;
  int cur = 0;
  long long launches = 0;
  int prof_group = 0;  // 0 = off, else the kernel group timed with events
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  StepGraph graphs[2];
  bool use_graph = true;
  cudaStream_t cap_st = nullptr;
};

struct mr_lbm_batch;

struct mr_lbm : Exec {
  Geo g;
  MeshDev mesh[2];
  MeshCounts* cntbuf = nullptr;  // two MeshCounts
  void* fstate = nullptr;    // leaf populations [Q][cap_leaf], storage type of the form
  void* fscratch = nullptr;  // pre-transport leaf populations, same layout
  uint8_t* flags = nullptr;
  uint8_t* cls = nullptr;
  uint8_t* act = nullptr;  // two bytes per dense chunk: InstDev::act, then InstDev::acth
  int* bcounts = nullptr;
  int32_t* inidx = nullptr;
  unsigned long long* vol = nullptr;
  double* W = nullptr;
  float* Wf = nullptr;
  double* Ws = nullptr;  // s = 2, 3: flattened weights of half-width 2s
  void* det = nullptr;   // D2Q9, s = 1: critical-case details (see InstDev::det)
  float* Wsf = nullptr;
  double* dense[2] = {nullptr, nullptr};
  size_t dense_elems = 0;
  void* staging = nullptr;
  size_t staging_bytes = 0;
  // upload of mr_lbm_set_leaves' populations beside the mesh build
  cudaStream_t up_st = nullptr;
  cudaEvent_t ev_prior = nullptr, ev_up = nullptr;
  bool initialized = false;
  mr_status sticky = MR_OK;
  std::vector<void*> allocs;
  // The instance's descriptor in device memory (its slot in the batch's
  // array when it belongs to a batch) and the group of one that the
  // single-instance calls launch with.
  InstDev* dinst = nullptr;
  Group grp;
  mr_lbm_batch* batch = nullptr;
};

// Record a sticky failure on the handle and return it.
mr_status mr_handle_fail(mr_lbm* h, mr_status s);
// Queue the bottom-up projection of the current state into the internal
// cells of the current mesh (no allocation).
void mr_handle_projection(mr_lbm* h);
// Copy both meshes' counters to the host, synchronise, and turn device error
// bits into a status (no allocation).
mr_status mr_handle_read_counts(mr_lbm* h, MeshCounts* out /*[2]*/);
