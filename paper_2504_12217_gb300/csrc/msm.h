// Pippenger multi-scalar multiplication engine (internal).
#pragma once
#include <vector>

#include "curve.cuh"
#include "internal.h"

namespace zkvc {

enum ScalarKind : int32_t {
  SK_ONE = 0,       // the scalar 1 (no array)
  SK_I8 = 1,        // int8 array, signed
  SK_I32 = 2,       // int32 array, signed, |v| < 2^31
  SK_FR_MONT = 3,   // Fr array in Montgomery form
  SK_FR_CANON = 4,  // Fr array, canonical little-endian 8 x u32
  SK_I16 = 5,       // int16 array, signed
  SK_SIGNED127 = 6, // uint4 array: magnitude < 2^127 in bits 0..126, sign in bit 127
};

// One run of points sharing a scalar kind and an output.
struct MsmSeg {
  uint64_t base_off;   // index of window 0 of point 0 in the base array
  uint32_t count;      // points
  uint32_t nwin;       // bases stored per point: 2^(c w) multiples for w < nwin
  uint32_t out;        // output index
  int32_t kind;        // ScalarKind
  const void* scalars; // device array (unused for SK_ONE)
  uint32_t skip;       // point whose scalar is ignored (0xffffffff: none)
  uint32_t nd;         // digits per scalar (planner)
  uint64_t slot_off;   // first digit slot (planner)
  uint32_t point_off;  // cumulative points before this segment (planner)
  uint32_t pad;
};

struct MsmOut {
  uint32_t c;          // window bits; digit magnitudes 1 .. 2^(c-1)
  uint32_t win_keys;   // >1: windows get their own buckets (variable base) and are
                       // combined by Horner's rule; 1: windows use precomputed bases
  uint32_t key_off;    // planner
  uint32_t nkeys;      // planner: win_keys * 2^(c-1)
  const void* bases;   // this output's base array (nullptr: the run's), so one run can
                       // serve outputs of several proving keys
};

// Launch-shape knobs of a run (chosen by the batch autotuner; defaults otherwise).
struct MsmTune {
  uint32_t chunk = 0;          // terms per level-0 chunk (0: the default rule of msm_plan_finalize)
  uint32_t accum_threads = 128;
  uint32_t lanes = 0;          // lanes per chunk: 1, 4 (a quad), 0 = by the run's size
};

struct MsmPlan {
  MsmTune tune;
  std::vector<MsmSeg> segs;
  std::vector<MsmOut> outs;
  uint64_t slots = 0;
  uint32_t keys = 0;
  uint32_t points = 0;
  uint32_t max_nd = 0;
  uint32_t chunk = 0;          // planner: the level-0 chunk in use
  uint32_t lanes = 1;          // planner: lanes per chunk in use
  int32_t key_shift = -1;      // planner: log2 of the keys per output when outputs carry
                               // their own bases (all outputs then have equal 2^k keys)
};

// Fills the planner fields; returns ZKVC_EINVAL on an inconsistent plan.
int msm_plan_finalize(MsmPlan& p);

// Device workspace the run needs (bytes), for a finalized plan and coordinate field.
template <class F>
size_t msm_workspace_bytes(const MsmPlan& p);

// Runs every output of the plan; results[o] receives output o (XYZZ, device).  If
// after_accum is given it is recorded on `st` once the bucket accumulation is enqueued
// (other streams may wait for the end of the run's throughput-bound part).
template <class F>
int msm_run(const MsmPlan& p, const Affine<F>* bases, void* ws, size_t ws_bytes, XYZZ<F>* results,
            cudaStream_t st, int accum_stage = -1, cudaEvent_t after_accum = nullptr);

// The same run split in three, for launch sequences that are built once and replayed
// (CUDA graphs): prepare carves the workspace and builds the host tables, upload copies
// the tables to their place in the workspace (host -> device; not under capture), and
// launch issues only kernels, memsets and device copies (capturable).  The plan's scalar
// and base pointers are baked into the uploaded tables.
struct MsmExecState;
struct MsmExec {
  MsmPlan plan;
  MsmExecState* st = nullptr;
  MsmExec() = default;
  MsmExec(const MsmExec&) = delete;
  MsmExec& operator=(const MsmExec&) = delete;
  ~MsmExec();
};
template <class F>
int msm_prepare(const MsmPlan& p, void* ws, size_t ws_bytes, MsmExec* ex);
int msm_upload(MsmExec* ex, cudaStream_t st);
// While set (this thread), msm_upload writes its table images into the pinned host
// buffer [host, host + cap) instead of temporary memory: for uploads captured into a
// graph, whose copy nodes read the images again on every replay.  nullptr unsets it.
void msm_table_stage(uint8_t* host, size_t cap);
template <class F>
int msm_launch(const MsmExec* ex, const Affine<F>* bases, XYZZ<F>* results, cudaStream_t st, int accum_stage = -1,
               cudaEvent_t after_accum = nullptr);
// Device address of the run's bucket-term count (valid after a launch completes).
const uint32_t* msm_term_count(const MsmExec* ex);

// The variable-base MSM behind zkvc_msm_g1 / zkvc_msm_g2: canonical points and scalars
// in, canonical affine result out (host), using the caller's workspace.
template <class F>
int msm_api(const uint8_t* d_points, const uint8_t* d_scalars, size_t n, void* d_ws, size_t ws_bytes,
            uint8_t* out, cudaStream_t st);
template <class F>
size_t msm_api_ws(size_t n);

// Exclusive scan of n uint32 values into out[0..n] (out[n] = total); temp from the arena;
// copy (if non-null) receives out[0..n) as well.
int scan_u32(const uint32_t* in, uint32_t* out, size_t n, Arena& a, cudaStream_t st, uint32_t* copy = nullptr);
size_t scan_u32_temp_bytes(size_t n);

}  // namespace zkvc
