// Planner kernels, one per step of the batch-synchronous iteration, and their
// launchers (single problem and batched form); the device code of every step
// lives in stp_planner_body.cuh, shared with the persistent planner kernel.
#include "stp_planner_body.cuh"

namespace stp {

// ---------------------------------------------------------------------------
// Kernels: single problem (structs as parameters) and batch (problem
// blockIdx.y, structs staged in shared memory).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_reset(State<R> S, int max_iters) { reset_body(S, max_iters); }
template <typename R>
__global__ void __launch_bounds__(kSampleThreads) k_sample(Geom<R> G, State<R> S) { sample_body(G, S, blockIdx.x, gridDim.x); }
template <typename R, int DQ>
__global__ void __launch_bounds__(kQT) k_nn(Geom<R> G, State<R> S) { nn_body<R, DQ>(G, S, blockIdx.x, gridDim.x); }
template <typename R>
__global__ void __launch_bounds__(kCtaThreads) k_insert(Geom<R> G, State<R> S) { insert_body(G, S); }
template <typename R, int DQ>
__global__ void __launch_bounds__(kQT) k_bridge(Geom<R> G, State<R> S) { bridge_body<R, DQ>(G, S, blockIdx.x, gridDim.x); }
template <typename R>
__global__ void __launch_bounds__(kCtaThreads) k_publish(Geom<R> G, State<R> S) { publish_body(G, S); }
template <typename R>
__global__ void k_extract_path(State<R> S) { extract_path_body(S); }

template <typename R>
__global__ void k_reset_b(const State<R>* Ss, const int* max_iters) {
    __shared__ Geom<R> G;
    __shared__ State<R> S;
    stage_problem((const Geom<R>*)nullptr, Ss, blockIdx.y, G, S, false);
    reset_body(S, max_iters[blockIdx.y]);
}
template <typename R>
__global__ void __launch_bounds__(kSampleThreads) k_sample_b(const Geom<R>* Gs, const State<R>* Ss) {
    __shared__ Geom<R> G;
    __shared__ State<R> S;
    stage_problem(Gs, Ss, blockIdx.y, G, S);
    sample_body(G, S, blockIdx.x, gridDim.x);
}
template <typename R, int DQ>
__global__ void __launch_bounds__(kQT) k_nn_b(const Geom<R>* Gs, const State<R>* Ss) {
    __shared__ Geom<R> G;
    __shared__ State<R> S;
    stage_problem(Gs, Ss, blockIdx.y, G, S);
    nn_body<R, DQ>(G, S, blockIdx.x, gridDim.x);
}
// Batched single-CTA steps run NT threads a problem: 256 when no problem has
// more workers (one insertion round, eight CTAs an SM), else 1024.
template <typename R, int NT>
__global__ void __launch_bounds__(NT) k_insert_b(const Geom<R>* Gs, const State<R>* Ss) {
    __shared__ Geom<R> G;
    __shared__ State<R> S;
    stage_problem(Gs, Ss, blockIdx.y, G, S);
    insert_body<R, NT>(G, S);
}
template <typename R, int DQ>
__global__ void __launch_bounds__(kQT) k_bridge_b(const Geom<R>* Gs, const State<R>* Ss) {
    __shared__ Geom<R> G;
    __shared__ State<R> S;
    stage_problem(Gs, Ss, blockIdx.y, G, S);
    bridge_body<R, DQ>(G, S, blockIdx.x, gridDim.x);
}
template <typename R, int NT>
__global__ void __launch_bounds__(NT) k_publish_b(const Geom<R>* Gs, const State<R>* Ss) {
    __shared__ Geom<R> G;
    __shared__ State<R> S;
    stage_problem(Gs, Ss, blockIdx.y, G, S);
    publish_body(G, S);
}
template <typename R>
__global__ void k_extract_path_b(const State<R>* Ss) {
    __shared__ Geom<R> G;
    __shared__ State<R> S;
    stage_problem((const Geom<R>*)nullptr, Ss, blockIdx.y, G, S, false);
    extract_path_body(S);
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
const char* const kIterKernelNames[kIterKernels] = {"k_sample", "k_nn", "k_validate(ext)", "k_insert",
                                                    "k_bridge", "k_validate(bridge)", "k_publish"};

template <typename R>
cudaError_t launch_plan_reset(const Geom<R>& g, const State<R>& s, int max_iters, cudaStream_t st) {
    k_reset<R><<<1, 256, 0, st>>>(s, max_iters);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_iteration(const Geom<R>& g, const State<R>& s, int vgrid, cudaStream_t st, cudaEvent_t* ev) {
    const int nn_grid = 4 * validate_grid_blocks();
    const int wgrid = (s.W + kSampleThreads - 1) / kSampleThreads;
    int ne = 0;
    // External event-record nodes: inside a stream capture a plain event record
    // only adds a dependency edge and cannot be timed.
    auto mark = [&]() {
        if (ev) cudaEventRecordWithFlags(ev[ne], st, cudaEventRecordExternal);
        ++ne;
    };
    mark();
    k_sample<R><<<wgrid, kSampleThreads, 0, st>>>(g, s);
    mark();
    // Coordinates beyond the problem's DOF are zero in every node and query,
    // so a narrower scan gives the same keys.
    if (g.dof <= 3) k_nn<R, 3><<<nn_grid, kQT, 0, st>>>(g, s);
    else if (g.dof == 6) k_nn<R, 6><<<nn_grid, kQT, 0, st>>>(g, s);
    else k_nn<R, kMaxDof><<<nn_grid, kQT, 0, st>>>(g, s);
    mark();
    cudaError_t err = launch_validate<R>(g, ext_batch(s), false, true, vgrid, st);
    if (err != cudaSuccess) return err;
    mark();
    k_insert<R><<<1, kCtaThreads, 0, st>>>(g, s);
    mark();
    if (g.dof <= 3) k_bridge<R, 3><<<nn_grid, kQT, 0, st>>>(g, s);
    else if (g.dof == 6) k_bridge<R, 6><<<nn_grid, kQT, 0, st>>>(g, s);
    else k_bridge<R, kMaxDof><<<nn_grid, kQT, 0, st>>>(g, s);
    mark();
    // Bridges are long: a coarse pass over every eighth check point finds most
    // collisions, then only the entries it left free are checked in full.
    {
        EdgeBatch<R> bb = bridge_batch(s);
        bb.phase = 1;
        err = launch_validate<R>(g, bb, false, true, vgrid, st);
        if (err != cudaSuccess) return err;
        bb.phase = 2;
        err = launch_validate<R>(g, bb, false, true, vgrid, st);
        if (err != cudaSuccess) return err;
    }
    mark();
    k_publish<R><<<1, kCtaThreads, 0, st>>>(g, s);
    mark();
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_extract_path(const State<R>& s, int dof, cudaStream_t st) {
    k_extract_path<R><<<1, 64, 0, st>>>(s);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_plan_reset_batch(const State<R>* Ss, const BatchShape& b, const int* max_iters, cudaStream_t st) {
    k_reset_b<R><<<dim3(1, b.P), 256, 0, st>>>(Ss, max_iters);
    return cudaGetLastError();
}

// One batched iteration: every kernel covers all problems (grid y = problem).
// Mixed degrees of freedom use the 7-coordinate NN key (missing coordinates
// are zero) and a run-time arm/point choice in the collision kernel.
template <typename R>
cudaError_t launch_iteration_batch(const Geom<R>* Gs, const State<R>* Ss, const BatchShape& b, cudaStream_t st) {
    const int wgrid = (b.max_W + kSampleThreads - 1) / kSampleThreads;
    k_sample_b<R><<<dim3(wgrid, b.P), kSampleThreads, 0, st>>>(Gs, Ss);
    k_nn_b<R, kMaxDof><<<dim3(b.nn_ctas, b.P), kQT, 0, st>>>(Gs, Ss);
    cudaError_t err = launch_validate_batch<R>(Gs, Ss, b.P, 0, b.max_obs, b.validate_ctas, b.validate_smem, st);
    if (err != cudaSuccess) return err;
    const bool narrow = b.max_W <= 256;
    if (narrow) k_insert_b<R, 256><<<dim3(1, b.P), 256, 0, st>>>(Gs, Ss);
    else k_insert_b<R, kCtaThreads><<<dim3(1, b.P), kCtaThreads, 0, st>>>(Gs, Ss);
    k_bridge_b<R, kMaxDof><<<dim3(b.nn_ctas, b.P), kQT, 0, st>>>(Gs, Ss);
    err = launch_validate_batch<R>(Gs, Ss, b.P, 1, b.max_obs, b.validate_ctas, b.validate_smem, st);
    if (err != cudaSuccess) return err;
    err = launch_validate_batch<R>(Gs, Ss, b.P, 2, b.max_obs, b.validate_ctas, b.validate_smem, st);
    if (err != cudaSuccess) return err;
    if (narrow) k_publish_b<R, 256><<<dim3(1, b.P), 256, 0, st>>>(Gs, Ss);
    else k_publish_b<R, kCtaThreads><<<dim3(1, b.P), kCtaThreads, 0, st>>>(Gs, Ss);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_extract_path_batch(const State<R>* Ss, const BatchShape& b, cudaStream_t st) {
    k_extract_path_b<R><<<dim3(1, b.P), 64, 0, st>>>(Ss);
    return cudaGetLastError();
}

template cudaError_t launch_plan_reset_batch<float>(const State<float>*, const BatchShape&, const int*, cudaStream_t);
template cudaError_t launch_iteration_batch<float>(const Geom<float>*, const State<float>*, const BatchShape&,
                                                   cudaStream_t);
template cudaError_t launch_extract_path_batch<float>(const State<float>*, const BatchShape&, cudaStream_t);

template cudaError_t launch_plan_reset<float>(const Geom<float>&, const State<float>&, int, cudaStream_t);
template cudaError_t launch_plan_reset<double>(const Geom<double>&, const State<double>&, int, cudaStream_t);
template cudaError_t launch_iteration<float>(const Geom<float>&, const State<float>&, int, cudaStream_t,
                                            cudaEvent_t*);
template cudaError_t launch_iteration<double>(const Geom<double>&, const State<double>&, int, cudaStream_t,
                                             cudaEvent_t*);
template cudaError_t launch_extract_path<float>(const State<float>&, int, cudaStream_t);
template cudaError_t launch_extract_path<double>(const State<double>&, int, cudaStream_t);

}  // namespace stp
