// sfac_batch_launch.h - host entry points of the batch kernels (one
// translation unit per precision) and the schedule they consume.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "sfac.h"

namespace sfac {

// One instance as the persistent kernel sees it.
struct BatchInst {
    void* u;                // field (device), layout of PassArgs
    long long npts;
    int dim;
    int steps;              // steps of this run
    int n[3];
    int items[3];           // work items of one pass along each axis
    const void* tab[3][2];  // per axis: eC, eS (see PassArgs); twists and twiddles: BatchSchedule::common
    double jq[4];           // e^{-tau}, 1 - e^{-tau}, e^{-2 tau}, 1 - e^{-2 tau}
};

struct BatchSchedule {
    const BatchInst* inst;
    const long long* phase_base;   // [nphase + 1] number of the first item of each phase
    const int* phase_step;         // [nphase]
    const int* phase_axis;         // [nphase]
    const long long* phase_first;  // [nphase + 1] first slot of each phase
    const int* slot_inst;          // instance of each slot (phase, active instance)
    const long long* slot_cum;     // inclusive running sum of items within the phase
    int nphase;
    int mult;                      // warp-groups per item
    long long total_items;
    unsigned long long* counter;   // next item to claim
    unsigned long long* done;      // [ninst] items completed per instance
    int* error;                    // 0, or SFAC_BATCH_TIMEOUT
    long long spin_limit;          // polls before a wait gives up
    int hold_instance;             // test hook: this instance's second pass never becomes ready (-1: off)
    const void* common;            // twiddles and twists of every length (batch_common_offset), precision R
    int stage;                     // > 0: strided items are staged in shared memory (= mult; FP32 only)
};

// Staging buffer of one warp for strided items (see sfac_batch.cuh), in
// complex values: the item's lines (mult * 32/T of them, 512 * mult values for
// 16 values per thread) with BATCH_STAGE_PAD values of padding each.
constexpr int BATCH_STAGE_PAD = 2;
__host__ __device__ constexpr int batch_stage_elems(int mult) { return 544 * mult; }

// Twiddles e^{-2 pi i k/N} and twists e^{i pi k/N} depend on the line length
// only. One device block holds them for N = 32 .. 512, as complex values of the
// batch's precision: at batch_common_offset(N) the N twiddles, then the N
// twists. Each CTA of the batch kernel copies the block into shared memory.
constexpr int BATCH_COMMON_ELEMS = 2 * (32 + 64 + 128 + 256 + 512);
__host__ __device__ constexpr int batch_common_offset(int N) { return 2 * (N - 32); }

// Allocate and fill that block for precision `prec` (synchronous upload).
sfac_status make_common_tables(int prec, void** dev);

constexpr int SFAC_BATCH_TIMEOUT = 1;

// The persistent batch kernel with `wpb` warps per CTA (<= 8) and `es` values
// per thread for lines up to 256 points (8 or 16; FP64 always 16).
// setup_*: set its shared-memory limit and compute the persistent grid for
// `sms` SMs with staging buffers for `stage` warp-groups per item (0: none);
// call outside stream capture. launch_*: enqueue it on `s` (staging as in
// sc.stage, which must equal the `stage` given to setup).
// cudaErrorInvalidValue for other shapes.
cudaError_t setup_batch_f32(int wpb, int es, int stage, int sms, int* grid);
cudaError_t setup_batch_f64(int wpb, int es, int stage, int sms, int* grid);
cudaError_t launch_batch_f32(int wpb, int es, int grid, const BatchSchedule& sc, cudaStream_t s);
cudaError_t launch_batch_f64(int wpb, int es, int grid, const BatchSchedule& sc, cudaStream_t s);

// Items per pass of every axis of I for a kernel shape with `es` values per
// thread below N = 512 and `mult` warp-groups per item.
void set_items(BatchInst& I, int es, int mult);

// Byte offsets of the seven arrays of a packed schedule (instances,
// phase_base, phase_first, slot_cum, phase_step, phase_axis, slot_inst), its
// size and counts.
struct ScheduleLayout {
    size_t off[7];
    size_t total;
    int nphase;
    long long total_items;
};

// Build the phase schedule of `inst` (fields, steps and items set) into `blob`
// (host memory, resized to lay->total bytes).
void pack_schedule(const std::vector<BatchInst>& inst, std::vector<unsigned char>& blob, ScheduleLayout* lay);
// Point the schedule arrays of `sc` into a device copy of a packed blob at `dev`
// (its scratch pointers, spin limit, hold instance, common tables and staging
// are left as they are).
void bind_schedule(const ScheduleLayout& lay, void* dev, int mult, BatchSchedule* sc);

// Build the phase schedule of `inst` (fields, steps and items set) and upload
// it into *dev (grown as needed, *cap bytes); fills `sc` except its scratch
// pointers, spin limit and hold instance. Synchronises `st`.
sfac_status upload_schedule(const std::vector<BatchInst>& inst, int mult, void** dev, size_t* cap,
                            BatchSchedule* sc, cudaStream_t st);

// Kernel shape `index` of the batch autotuner's list (false if out of range).
bool batch_shape(int index, int* wpb, int* es, int* mult);

}  // namespace sfac
