// Persistent planner kernel: arguments and host launchers (stp_persist.cu).
#pragma once

#include "stp_internal.cuh"

namespace stp {

// Each team's barrier counter sits in a 128-byte line of its own.
constexpr int kPersistSyncStride = 32;

// Scratch of one persistent launch (device memory, zeroed before the launch):
// team barrier counters [teams][kPersistSyncStride], the problem queue, the
// problem each team plans, and the flag that stops every team when a barrier
// wait ran out.
struct PersistScratch {
    unsigned* sync;
    int* queue;
    int* team_prob;
    int* abort_flag;
};

constexpr size_t persist_scratch_bytes(int teams) {
    return sizeof(unsigned) * (size_t)teams * kPersistSyncStride + sizeof(int) * (size_t)(teams + 2);
}

template <typename R>
struct PersistArgs {
    const Geom<R>* Gs;     // [P] problems' geometry (device)
    const State<R>* Ss;    // [P] problems' state (device)
    const int* max_iters;  // [P] iteration budgets (device)
    int P;                 // problems
    int team_size;         // CTAs per team (the grid is a whole number of teams)
    unsigned* sync;
    int* queue;
    int* team_prob;
    int* abort_flag;
};

int persist_dq(int max_dof);
// Dynamic shared memory of a launch: the largest geometry blob and the
// collision batch's offsets (2 W + 1 ints).
int persist_smem_bytes(int max_blob_bytes, int max_W);
// Threads of a persistent CTA: the batch queue's (FP32 only) or a lone problem's.
int persist_threads(bool batch);
template <typename R>
cudaError_t persist_blocks_per_sm(int dq, int smem, int* blocks, int threads);
// Cooperative launch of grid CTAs of `threads` threads (persist_threads);
// grid <= 0 only configures the kernel's shared-memory limit.
template <typename R>
cudaError_t launch_plan_persistent(const PersistArgs<R>& a, int dq, int grid, int smem, cudaStream_t st, int threads);

}  // namespace stp
