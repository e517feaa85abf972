// Persistent planner kernel: a whole plan (reset, every batch-synchronous
// iteration of Algorithm 1 inside Algorithm 2 or 3, path extraction) in one
// launch, for one problem or for a batch of problems.
//
// The grid is split into teams of CTAs that are resident together (a
// cooperative launch checks it). A team plans one problem at a time; with a
// batch, each team takes the next problem from a device work queue when it
// finishes the previous one. Within a team the steps of an iteration run in
// order, separated by team barriers (an arrival counter in global memory and a
// bounded spin on it) instead of kernel boundaries:
//   sample -> NN + steer -> validate extensions -> insert -> bridge scan ->
//   validate bridges (coarse, then full) -> publish / allocation update.
// Every CTA keeps the problem's geometry blob in shared memory for the whole
// plan (one TMA bulk copy per problem). The single-CTA steps (insert, publish)
// run on the team's first CTA while the others wait at the next barrier. The
// step bodies are the ones of the per-step kernels (stp_planner_body.cuh,
// stp_validate_body.cuh): the same arithmetic in the same order, so results
// equal the per-step kernels' bit for bit.
//
// Every barrier wait is bounded by 1 s of global time: a team whose wait runs
// out sets the plan's error flag (STP_ERR_TIMEOUT) and its CTAs return.
#include "stp_persist.cuh"
#include "stp_planner_body.cuh"
#include "stp_validate_body.cuh"

namespace stp {

// CTA sizes: 512 threads for a lone problem (one CTA an SM, every CTA on the
// problem's team); 256 for the batch queue (two CTAs an SM, so two teams share
// an SM and one computes while the other waits at a barrier).
constexpr int kPersistThreads = 512, kPersistBatchThreads = 256;
constexpr int kPhases = 8;

// Team barrier (sense reversal on one word). Each barrier adds exactly 2^31
// to the team's counter: the team's first CTA adds 2^31 - (size - 1), every
// other CTA adds 1, so bit 31 of the counter flips when, and only when, the
// last arrival lands. Every CTA remembers the value its own arrival returned
// and polls the word until that bit differs. Thread 0 fences before arriving
// (release) and after the wait (acquire), so the team's writes before the
// barrier are visible after it. Returns false (and raises *abort) when the
// wait runs out, or when another CTA has raised *abort.
__device__ __forceinline__ bool team_sync(unsigned* counter, bool first, unsigned size, int* abort_flag) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned add = first ? 0x80000000u - (size - 1u) : 1u;
        __threadfence();
        const unsigned old = atomicAdd(counter, add);
        int ok = 1;
        const unsigned long long t0 = global_ns();
        for (unsigned it = 0;; ++it) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(counter) : "memory");
            if ((v ^ old) & 0x80000000u) break;
            if ((it & 63u) == 63u) {
                if (*(volatile int*)abort_flag) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > kWaitLimitNs) {
                    atomicExch(abort_flag, 1);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename R, int MO>
__device__ __forceinline__ void validate_step(const Geom<R>& G, const EdgeBatch<R>& E, unsigned char* smem, int cta,
                                              int ncta) {
    if (G.arm) validate_body<R, true, MO, false, true>(G, E, smem, cta, ncta, true);
    else validate_body<R, false, MO, false, true>(G, E, smem, cta, ncta, true);
}

template <typename R, int DQ, int MO, int NT>
__global__ void __launch_bounds__(NT, kPersistThreads / NT)
    k_plan_persistent(const __grid_constant__ PersistArgs<R> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Geom<R> G;
    __shared__ State<R> S;
    __shared__ __align__(8) uint64_t blob_bar;
    __shared__ int s_prob;
    const int team = (int)blockIdx.x / A.team_size;
    const int rank = (int)blockIdx.x % A.team_size;
    const int ts = A.team_size;
    unsigned* counter = A.sync + (size_t)team * kPersistSyncStride;
    const bool first = rank == 0;
    if (threadIdx.x == 0) mbar_init(&blob_bar, 1);
    __syncthreads();
    unsigned blob_phase = 0;
    for (int round = 0;; ++round) {
        // Next problem: the team's first CTA takes it from the queue.
        if (threadIdx.x == 0 && rank == 0) A.team_prob[team] = A.P > 1 ? atomicAdd(A.queue, 1) : round;
        if (!team_sync(counter, first, ts, A.abort_flag)) return;
        if (threadIdx.x == 0) s_prob = *(volatile int*)&A.team_prob[team];
        __syncthreads();
        const int p = s_prob;
        if (p >= A.P) return;
        stage_problem(A.Gs, A.Ss, p, G, S);  // ends with __syncthreads
        // The geometry blob stays in shared memory for the whole plan.
        if (threadIdx.x == 0) {
            mbar_expect_tx(&blob_bar, G.blob_bytes);
            bulk_g2s(smem_raw, G.blob, G.blob_bytes, &blob_bar);
        }
        if (!mbar_wait(&blob_bar, blob_phase)) {
            if (threadIdx.x == 0) {
                atomicOr(&S.ctl->err, kErrTimeout);
                atomicExch(A.abort_flag, 1);
            }
            return;
        }
        blob_phase ^= 1u;
        if (rank == 0) reset_body(S, A.max_iters[p]);
        if (!team_sync(counter, first, ts, A.abort_flag)) break;
        unsigned long long t_prev = global_ns();
        auto step_done = [&](int phase) -> bool {
            const bool ok = team_sync(counter, first, ts, A.abort_flag);
            if (ok && rank == 0 && threadIdx.x == 0) {
                const unsigned long long now = global_ns();
                S.ctl->ph_ns[phase] += now - t_prev;
                t_prev = now;
            }
            return ok;
        };
        bool ok = true;
        while (ok) {
            if (*(volatile int*)&S.ctl->done) break;
            sample_body(G, S, rank, ts);
            if (!(ok = step_done(0))) break;
            nn_body<R, DQ, NT / kQT>(G, S, rank, ts);
            if (!(ok = step_done(1))) break;
            validate_step<R, MO>(G, ext_batch(S), smem_raw, rank, ts);
            if (!(ok = step_done(2))) break;
            if (rank == 0) insert_body<R, NT>(G, S);
            if (!(ok = step_done(3))) break;
            bridge_body<R, DQ, NT / kQT>(G, S, rank, ts);
            if (!(ok = step_done(4))) break;
            // Bridges are long: a coarse pass over every eighth check point
            // finds most collisions, then the entries it left free in full.
            EdgeBatch<R> bb = bridge_batch(S);
            bb.phase = 1;
            validate_step<R, MO>(G, bb, smem_raw, rank, ts);
            if (!(ok = step_done(5))) break;
            bb.phase = 2;
            validate_step<R, MO>(G, bb, smem_raw, rank, ts);
            if (!(ok = step_done(6))) break;
            if (rank == 0) publish_body(G, S);
            if (!(ok = step_done(7))) break;
        }
        if (!ok) {
            if (threadIdx.x == 0) {
                atomicOr(&S.ctl->err, kErrTimeout);
                atomicExch(&S.ctl->done, 1);
            }
            return;
        }
        if (rank == 0) extract_path_body(S);  // the first CTA, every thread
    }
}

// One shared-memory record per kernel instance, used by launches and
// occupancy queries alike (the attribute only ever grows).
template <typename R, int DQ, int MO, int NT>
static SmemAttr& attr_pk() {
    static SmemAttr attr;
    return attr;
}

template <typename R, int DQ, int MO, int NT>
static cudaError_t launch_pk(const PersistArgs<R>& a, int grid, int smem, cudaStream_t st) {
    auto kern = k_plan_persistent<R, DQ, MO, NT>;
    cudaError_t e = ensure_smem((const void*)kern, attr_pk<R, DQ, MO, NT>(), smem);
    if (e != cudaSuccess) return e;
    if (grid <= 0) return cudaSuccess;  // configuration only
    void* args[] = {const_cast<PersistArgs<R>*>(&a)};
    return cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(NT), args, (size_t)smem, st);
}

template <typename R, int DQ, int MO, int NT>
static cudaError_t occupancy_pk(int smem, int* blocks) {
    auto kern = k_plan_persistent<R, DQ, MO, NT>;
    cudaError_t e = ensure_smem((const void*)kern, attr_pk<R, DQ, MO, NT>(), smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, NT, smem);
}

template <typename R, int DQ, int MO, int NT>
static cudaError_t run_pk(const PersistArgs<R>* a, int grid, int smem, cudaStream_t st, int* blocks) {
    return blocks ? occupancy_pk<R, DQ, MO, NT>(smem, blocks) : launch_pk<R, DQ, MO, NT>(*a, grid, smem, st);
}

// Kernel variants: FP32 with 3, 6 or 7 coordinates in the NN keys (point
// robots, six-axis and seven-axis arms) and 16-obstacle register chunks at 512
// threads, and the batch queue's 7-coordinate variant at 256 threads; FP64
// (the parity mode) with 7 coordinates (missing ones are zero in nodes and
// queries, so the keys are the same) and 8-obstacle chunks.
template <typename R>
static cudaError_t dispatch(int dq, int nt, const PersistArgs<R>* a, int grid, int smem, cudaStream_t st,
                           int* blocks) {
    if constexpr (sizeof(R) == 8) {
        return run_pk<R, 7, 8, kPersistThreads>(a, grid, smem, st, blocks);
    } else {
        if (nt == kPersistBatchThreads) return run_pk<R, 7, 16, kPersistBatchThreads>(a, grid, smem, st, blocks);
        if (dq <= 3) return run_pk<R, 3, 16, kPersistThreads>(a, grid, smem, st, blocks);
        if (dq == 6) return run_pk<R, 6, 16, kPersistThreads>(a, grid, smem, st, blocks);
        return run_pk<R, 7, 16, kPersistThreads>(a, grid, smem, st, blocks);
    }
}

int persist_dq(int max_dof) { return max_dof <= 3 ? 3 : (max_dof == 6 ? 6 : 7); }
int persist_smem_bytes(int max_blob_bytes, int max_W) {
    return ((max_blob_bytes + 15) / 16) * 16 + (int)sizeof(int) * (2 * max_W + 1);
}

int persist_threads(bool batch) { return batch ? kPersistBatchThreads : kPersistThreads; }

template <typename R>
cudaError_t persist_blocks_per_sm(int dq, int smem, int* blocks, int threads) {
    *blocks = 0;
    return dispatch<R>(dq, threads, nullptr, 0, smem, nullptr, blocks);
}

template <typename R>
cudaError_t launch_plan_persistent(const PersistArgs<R>& a, int dq, int grid, int smem, cudaStream_t st, int threads) {
    return dispatch<R>(dq, threads, &a, grid, smem, st, nullptr);
}

template cudaError_t persist_blocks_per_sm<float>(int, int, int*, int);
template cudaError_t persist_blocks_per_sm<double>(int, int, int*, int);
template cudaError_t launch_plan_persistent<float>(const PersistArgs<float>&, int, int, int, cudaStream_t, int);
template cudaError_t launch_plan_persistent<double>(const PersistArgs<double>&, int, int, int, cudaStream_t, int);

}  // namespace stp
