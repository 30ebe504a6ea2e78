// serve_internal.h -- the device-side layout of one serving step and the
// launchers of its kernels.  Not part of the public ABI.
//
// One step's tables are one contiguous buffer, written on the host and copied
// to the device before the step's graph runs:
//   StepHeader | TauLaunch[n_slots] | TauTask[n_tasks] | TauItem[n_items]
//              | RfSlot[n_rf] | RfUnit[n_units]
// (each table 16-byte aligned; offsets in the header).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lya_internal.h"

namespace lya {
namespace serve {

constexpr int kTauThreads = 1024;        // optical-depth CTA (one per SM)
constexpr int kTauMaxQ = 8;              // sources per thread: a group of 1024 >> s threads takes N <= 8192 >> s
constexpr int kMaxShift = 3;             // up to 8 skewers (warp groups) per CTA
constexpr int kRfThreads = 256;          // root-find CTA
constexpr int kRfRounds = 2;             // rounds of (Halley, Halley, flux) per step

struct StepHeader {
    unsigned int task_next;              // work counter of the optical-depth kernel (0 each step)
    int n_slots, n_tasks, n_items, n_rf, n_units;
    unsigned long long off_slots, off_tasks, off_items, off_rf, off_units;
};

struct TauTask {
    int slot;          // index into this step's TauLaunch table
    int first_item;    // items [first_item, first_item + n_items)
    int n_items;       // <= 1 << shift
    int shift;         // the CTA splits into 1 << shift warp groups
};

struct TauItem {
    long long src_row;     // skewer of the field
    long long out_row;     // row of the request's tau
};

struct RfSlot {
    const float* tau;
    float* flux;
    long long n;           // pixels
    double Ft, tol;
    int state;             // index of the request's root-find state and result
    int init;              // 1: first step of this root-find (state is reset)
    int unit_first, unit_count;
    int max_iter, pad;
};

struct RfUnit {
    int rf;                // index into this step's RfSlot table
    int pad;
    long long begin, end;  // pixels of the request's tau
};

// What the host reads back for each slot after a step.
struct SlotResult {
    double A, g;
    double m1, m2;                 // sums of (F - 1/2) and (F - 1/2)^2
    unsigned long long pdf[21];
    int iter, status, done, final; // final: the result is complete (F written, or failed)
};

template <typename T>
__host__ __device__ inline const T* step_table(const unsigned char* step, unsigned long long off)
{
    return reinterpret_cast<const T*>(step + off);
}

// Dynamic shared memory of the serving optical-depth CTA for one warp group
// on an n_pix, w_max skewer (16-byte multiple).
size_t serve_group_smem(int n_pix, int w_max);

// The serving optical-depth kernel: set its shared-memory limit (returns the
// dynamic bytes a CTA may use) and launch it over a step buffer.
cudaError_t serve_tau_prepare(size_t* dyn_smem);
cudaError_t serve_tau_launch(const unsigned char* d_step, size_t dyn_smem, int grid, cudaStream_t stream);

// Root-find state size (bytes) per slot, and the root-find passes of a step.
size_t serve_state_bytes();
cudaError_t serve_rf_launch(const unsigned char* d_step, void* d_states, SlotResult* d_results,
                            void* d_part, void* d_spart, int grid, cudaStream_t stream, int* n_launched);
size_t serve_part_bytes();
size_t serve_spart_bytes();

}  // namespace serve
}  // namespace lya
