// Device-resident plan and the apply entry points used by the C-ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "host.h"

namespace skel {

struct DeviceBuffers;   // per precision (defined in apply.cu)

struct DevicePlan {
    int device = 0;
    int dim = 3, kind = 1;
    double kappa = 0.0;
    bool cplx = false;
    int64_t N = 0, n_tot = 0;
    int nrhs_max = 32;
    int top = 1, L = 0;
    // shared index arrays (device)
    int64_t* box_off = nullptr;
    int32_t* box_n = nullptr;
    int32_t* box_nslot = nullptr;
    int32_t* slot_start = nullptr;
    int32_t* pos = nullptr;
    int64_t* eop = nullptr;                // user point -> its leaf entry
    int64_t* eop2 = nullptr;               // user point -> its skeleton row in the parent's slot, for
                                           // leaf boxes whose up/down steps the permutations do (-1: none;
                                           // null if no box qualifies)
    UpBox* up = nullptr;
    std::vector<int64_t> up_level_ptr;     // host copy
    std::vector<int32_t> up_level_maxk, up_level_maxr;   // per level: largest k, |I| - k
    int64_t* task_src = nullptr;
    uint64_t* task_mask = nullptr;
    int32_t* task_flags = nullptr;
    WorkItem* items = nullptr;
    int64_t n_items = 0;
    int64_t* part_ptr = nullptr;           // per entry: its partial sums (CUDA-core mode)
    int64_t* part_idx = nullptr;
    // tensor-core mode
    WorkItem* mix_items = nullptr;
    int64_t n_mix = 0;
    SrcTile* tc_tiles = nullptr;
    TcItem* tc_items = nullptr;
    int64_t n_tc = 0;
    int64_t tc_n_slots = 0;
    int64_t* tc_part_ptr = nullptr;        // per entry: its partial sums (tensor-core mode)
    int64_t* tc_part_idx = nullptr;
    int64_t* chunk_start = nullptr;        // source chunks (32 entries of one box)
    int32_t* chunk_cnt = nullptr;
    float* chunk_center = nullptr;         // 4 per chunk: its box's centre
    int64_t n_chunks = 0;
    float* tc_b = nullptr;                 // B operand per chunk for one 32-column pass (hi, lo)
    // stored-operator mode: store_mode 1 = per-tile store (every tile's
    // nrows x 32 values), 2 = symmetric store (shared blocks once); 0 = none
    int store_mode = 0;
    float* tc_a = nullptr;                 // the stored kernel values (either mode)
    int64_t* tc_abase = nullptr;           // per-tile store: per item, first float of its tiles
    std::vector<int64_t> tc_abase_host;
    uint8_t* tc_qmask = nullptr;           // per-tile store: per tile, the 4-column quads it keeps
    std::vector<uint8_t> tc_qmask_host;
    int64_t tile_floats = 0;               // floats the per-tile store takes
    void* tc_refs = nullptr;               // symmetric store: per tile and row chunk, BlockRef
    void* tc_isym = nullptr;               // symmetric store: per tensor-core item, ItemSym
    std::vector<unsigned char> tc_refs_host, tc_isym_host;  // the same on the host (kept to fill later)
    int64_t sym_floats = 0;                // floats the symmetric store takes
    int64_t pairs_stored = 0;              // kept kernel values the symmetric store holds once
                                           // (the rest are read transposed)
    int64_t n_tc_tiles = 0;
    int64_t stored_bytes = 0;              // 0 unless the tiles are stored
    // FP32 up/down launch shape per level: warps per CTA (0: the default
    // rule), set by the autotuner
    std::vector<int8_t> ud_warps_up, ud_warps_down;
    int tc_stages = 6;                     // bulk-copy stages of the on-the-fly tensor-core kernel (4, 6, 8)
    int tcs_stages = 4;                    // stages per CTA of the per-tile stored kernel (4 or 8)
    // tensor-core upward / downward passes (FP32_TC, real kernels): per
    // direction the work items (UdItem) grouped by level and their A blobs
    // FP32 T of the up/down boxes with columns padded to a multiple of 4
    // floats, 16-byte aligned per box (upward: k x (n - k), downward: the
    // transpose), and per box its first float (real kernels)
    float* ud_tp = nullptr;
    float* ud_ttp = nullptr;
    int64_t* ud_tp_off = nullptr;
    int64_t* ud_ttp_off = nullptr;
    // work lists of the CTA-wide up/down kernel: per direction (0 up, 1 down)
    // and rows per CTA (32 << i), (box, first row) pairs grouped by level
    int2* ud_work[2][4] = {{nullptr, nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr, nullptr}};
    std::vector<int64_t> ud_work_ptr[2][4];
    void* ud_items_up = nullptr;
    void* ud_items_down = nullptr;
    float* ud_a_up = nullptr;
    float* ud_a_down = nullptr;
    std::vector<int64_t> ud_ptr_up, ud_ptr_down;   // items of level l: [ptr[l], ptr[l + 1])
    int* status = nullptr;                 // device word raised by a bounded wait that gave up
    // test hook: the next tensor-core pass withholds its first item's first
    // tile until the compute warps gave up, with every wait limited to
    // test_wait_ns (skel_test_withhold_tile)
    bool test_withhold = false;
    uint64_t test_wait_ns = 0;
    DeviceBuffers* p64 = nullptr;
    DeviceBuffers* p32 = nullptr;
    // optional per-phase CUDA events (permute_in, up, near, reduce, down,
    // permute_out, end; then the start of the main translation kernel):
    // kProfEvents events for each of up to prof_cap applies
    std::vector<void*> events;
    int prof_cap = 0, prof_count = 0;
    std::vector<int> prof_launches, prof_main_launches;
    // host-pointer staging (allocated on first host-pointer call)
    void* stage_in = nullptr;
    void* stage_out = nullptr;
    size_t stage_bytes = 0;
    int64_t bytes = 0;
};

// Upload a layout; throws Error on failure. store_tiles: also evaluate every
// tensor-core tile's kernel values once and keep them (nrows x 128 B per tile), so
// that FP32_TC applies read them instead of evaluating (real kernels).
DevicePlan* device_plan_create(const Plan& p, const Layout& lay, int nrhs_max, int store_tiles = 0,
                               int store_stages = 4, bool updown_tc = false);
void device_plan_destroy(DevicePlan* dp);
// capture the phases of the next max_applies applies (0 = off)
void device_set_profiling(DevicePlan* dp, int max_applies);
// read and clear the device status word (synchronizes the device)
int device_status(DevicePlan* dp);
// summed milliseconds of the 6 phases over the captured applies (waits for them)
void device_last_timings(DevicePlan* dp, double* ms6, int* launches, int* n_applies, double* ms_main,
                         int* main_launches);

// Measure and keep the faster variants for FP32 applies of nrhs right-hand
// sides: per level the up/down kernel (plain or register prefetch), and,
// for the tensor-core path, on-the-fly or stored kernel tiles (stored only
// if allow_store and the tiles fit the free device memory). Synchronous;
// uses the plan's own buffers.
struct TuneReport {
    double ms_onfly = -1, ms_stored = -1;  // one tensor-core pass (bprep + translations)
    double ms_sym = -1;                     // the same reading the symmetric store (-1: not timed)
    int stored = 0;                         // store mode the plan keeps after tuning (0, 1, 2)
    int n_levels = 0, n_changed = 0;        // up/down launches timed, choices unlike the default rule
    double ms_updown_default = 0, ms_updown_tuned = 0;  // summed over the levels, one launch each
    int tc_stages = 0;                      // chosen pipeline depth of the on-the-fly kernel (0: not tuned)
    int tcs_stages = 0;                     // chosen stages per CTA of the per-tile stored kernel (0: not tuned)
};
TuneReport device_autotune(DevicePlan* dp, int nrhs, bool allow_store, void* stream);

// Allocation-failure test hook: the countdown-th allocation made through the
// library's helpers after this call fails as if memory were exhausted
// (0 = off). Returns true (and consumes the hook) when an allocation must fail.
void set_alloc_failure(int countdown);
bool alloc_should_fail();

// Algorithm 2 on `stream`. q, u: device pointers in user order (n x nrhs,
// each right-hand side contiguous). transpose: run with conj(T).
void device_apply(DevicePlan* dp, const void* q, void* u, int nrhs, int precision,
                  bool transpose, void* stream);

}  // namespace skel
