// Internal device-side definitions of the ST-pRRTC Extend library (sm_103a).
//
// Data layout in HBM (one problem):
//   geometry blob  spheres [S][4] (x,y,z,r; sorted by frame), waypoints
//                  [M][K][4] (t,x,y,z), segment velocities [M][K][4], radii [M]
//                  (padded to 4), waypoint times [M][8] (t_1..t_{K-1}, +inf
//                  padded); staged into shared memory by one TMA bulk copy
//                  per CTA in the collision kernel.
//   forward arena  SoA: x [cap_f][DP] (q..., zero pad, t at DP-1), parent, cost, iter.
//   backward arena N segments of cap_s nodes, same SoA plus troot and tree.
//   worker records SoA over W workers (sample, NN result, x_new, edge entries).
//   edge entries   SoA over <= 2W entries (root point checks, extensions,
//                  bridges): endpoints, check count c, prefix offsets, hit flag.
//   control block  Ctl: iteration counter, incumbent, allocation tables,
//                  slots, statistics.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

namespace stp {

// ---------------------------------------------------------------------------
// Host: per-device kernel configuration. Function attributes and SM counts
// belong to a device, so a process that uses several devices configures each
// one; a mutex guards the records against concurrent launches.
// ---------------------------------------------------------------------------
constexpr int kMaxDevices = 64;

struct SmemAttr {
    std::mutex mu;
    int bytes[kMaxDevices] = {};  // dynamic shared memory configured on each device
};

// Raises the kernel's dynamic shared-memory limit on the current device to at
// least smem bytes; *raised tells whether this call changed it.
inline cudaError_t ensure_smem(const void* kern, SmemAttr& a, int smem, bool* raised = nullptr) {
    if (raised) *raised = false;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(a.mu);
    if (smem <= a.bytes[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    a.bytes[dev] = smem;
    if (raised) *raised = true;
    return cudaSuccess;
}

constexpr int kMaxDof = 7;
constexpr int kDP = 8;          // padded node width for dof > 3
constexpr int kMaxRoots = 128;  // N
constexpr int kMaxSpheres = 64;
constexpr int kMaxObs = 128;
constexpr int kMaxWay = 8;
constexpr int kMaxWorkers = 8192;
constexpr int kQT = 128;        // queries per NN tile (= threads per CTA)
constexpr int kMaxTiles = 128;  // node tiles per query (FP64: partials per query)
constexpr int kMaxQTiles = kMaxWorkers / kQT;
constexpr int kNodeTileMin = 32;
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // bounded mbarrier waits: 1 s
constexpr unsigned kWaitLimit = 1u << 28;                   // and an iteration backstop
constexpr int kPropY = 160;                 // network output floats
constexpr int kPropSize = 24 + 16 * kMaxDof;
constexpr unsigned kThrLearned = 15099495u;  // learned iff m < ceil(0.9 2^24)

enum ErrBits { kErrCapacity = 1, kErrTimeout = 2, kErrInternal = 4 };

// ---------------------------------------------------------------------------
// Geometry (passed by value).
// ---------------------------------------------------------------------------
template <typename R>
struct Geom {
    int dof, arm, S, M, K, DP;
    int link_start[kMaxDof + 2];  // spheres of frame j: [link_start[j], link_start[j+1])
    R a[kMaxDof], d[kMaxDof], ca[kMaxDof], sa[kMaxDof], th0[kMaxDof];
    R qlo[kMaxDof], qhi[kMaxDof];
    R vmax;
    R ref[3];       // reference point subtracted from workspace positions in pair tests
    double vmax_d;  // v_max as given (edge check counts are evaluated in double)
    int continuous;  // point robots: closed-form edge validation
    int uniform_ro;  // every obstacle has the radius ro_uni
    R ro_uni;
    const R* blob;
    unsigned blob_bytes;
    int off_way, off_vel, off_rad, off_tim;  // offsets in R units inside the blob
    int off_self, n_self;  // self-collision pairs a * 64 + b (R values) and their count
};

// Flat batch of edges for the collision kernel. Entry e covers check points
// j = 1..cnt[e] at s = j / cnt[e] of (qa,ta) -> (qb,tb); point g of the flat
// range belongs to the entry with off[e] <= g < off[e+1].
template <typename R>
struct EdgeBatch {
    const R* qa;
    const R* qb;
    const R* ta;
    const R* tb;
    int qstride;             // R elements between consecutive edges' q
    const int* cnt;
    const long long* off;    // [n+1]
    const int* n_dev;        // device edge count (planner) or nullptr
    int n_host;
    int* hit;                // [n] 0/1
    R* clear;                // [n] (clearance mode) or nullptr
    unsigned long long* points_done;  // statistics or nullptr
    unsigned long long* pairs_done;   // executed sphere-obstacle pair tests or nullptr
    int* err;
    const int* done;                  // planner: skip the launch when set (or nullptr)
    // Precomputed-offset batches: window counter (device int, zero at launch)
    // from which CTAs take windows of consecutive edges as they finish the
    // previous one; nullptr deals the windows round-robin instead.
    int* win_next = nullptr;
    // In-kernel-scan batches only: 0 every check point; 1 the coarse subset
    // j = ceil((i+1) c / c0), i < c0 = ceil(c/8) (ends at j = c); 2 every
    // check point of the entries that phase 1 did not already find colliding.
    int phase = 0;
};

// ---------------------------------------------------------------------------
// Planner control block (device memory).
// ---------------------------------------------------------------------------
struct Ctl {
    int iter, done, err, pad0;
    int n_f, snap_f, n_trees, n_windows;
    int n_pieces, first_iter, inc_f, inc_s;
    int inc_b, max_iters, pad1, pad2;
    double U, C;
    // interval-root allocation (double)
    double Lg, H, dt, Ubar, width;
    int g_first[kMaxRoots], g_count[kMaxRoots];
    double g_meas[kMaxRoots];
    int group_active[kMaxRoots];
    // root-recycling slots
    double slot_T[kMaxRoots];
    long long slot_k[kMaxRoots];
    int slot_has[kMaxRoots], slot_active[kMaxRoots], slot_gen[kMaxRoots];
    // goal grid
    long long kmin, kend;  // checks kmin..kmin+nk-1; recycling roots in [kmin, kend)
    int nk, pad3;
    // per-segment counts
    int n_s[kMaxRoots], snap_s[kMaxRoots];
    // per-iteration NN bookkeeping
    int set_count[kMaxRoots + 1];
    int pad4, pad5, pad6, pad7;
    // statistics
    unsigned long long st_ext, st_bridge, st_root, st_ins, st_points, st_pairs;
    // scan work: (query, node) key evaluations and nodes read once per set
    unsigned long long st_nn_evals, st_nn_nodes, st_br_evals, st_br_nodes;
    unsigned long long t_start, t_first, t_end;
    // wall-clock budget of the plan in device global-timer ns (0: none),
    // checked after every iteration
    unsigned long long budget_ns;
    // persistent planner kernel: device time of each step (ns, summed over
    // iterations, measured barrier to barrier by the team's first CTA)
    unsigned long long ph_ns[8];
};

// Device pointers of one problem's planner state (passed by value).
template <typename R>
struct State {
    Ctl* ctl;
    int N, W, variant, cap_f, cap_s, cap_trees, max_pieces;
    double eta, res, p_new, p_guided, H;
    unsigned key0, key1, problem_id;
    // Coin thresholds on the 24-bit uniform m (u = m 2^-24):
    // guided iff m < thr_guided = ceil(p_guided 2^24); new root iff m <= thr_new = floor(p_new 2^24).
    unsigned thr_guided, thr_new;
    R qs[kMaxDof], qg[kMaxDof];
    // learned branch: table [kPropSize] = cumulative mixture weights (8), goal
    // time means (8) and standard deviations (8) in seconds, waypoints
    // [16][kMaxDof]; built from the network output prop_y [160].
    int learned;
    R* prop;
    float* prop_y;
    float* tgt;  // [131] training targets of the last path and a written flag
    // forward arena
    R* fx; int* fpar; R* fcost; int* fiter;
    // backward arena [N][cap_s]
    R* bx; int* bpar; R* bcost; R* btroot; int* btree; int* biter;
    // interval trees
    int* tree_group; double* tree_T;
    // allocation tables
    double* win_lo; double* win_hi; double* pc_lo; double* pc_hi; int* pc_group;
    // goal grid free flags [nk]
    unsigned char* gfree;
    // worker records [W]
    int* w_status; int* w_set; R* w_xr; R* w_T; int* w_parent; R* w_key; R* w_xnew;
    int* w_edge; int* w_root_edge; int* w_ins; int* w_bedge;
    R* w_xn;           // [W][kDP] steering source x_n
    unsigned long long* w_nnkey;  // [W] packed FP32 NN key (key bits << 32 | index)
    // NN
    int* qlist;        // [(N+1)][W]
    int* tile_cnt;     // [(N+1)][kMaxQTiles]
    R* part_k1; R* part_k2; int* part_idx;  // [W][kMaxTiles]
    // bridge
    int* bq_list;      // [2][W]: workers whose new node bridges to set 0 (fwd) / 1 (bwd concat)
    int* bq_count;     // [2]
    int* btile_cnt;    // [2][kMaxQTiles]
    unsigned long long* bkey;  // [W][2]: FP32 bridge rank (T_root, rho^2, index) packed in 128 bits
    int* b_set; int* b_idx; R* b_k1; R* b_k2;  // per worker best bridge candidate
    R* b_U; R* b_C;
    // edges
    R* eqa; R* eqb; R* eta_; R* etb; int* ecnt; int* ehit;  // [2W]: entry 2w root check, 2w+1 extension
    R* bqa; R* bqb; R* bta; R* btb; int* bcnt; int* bhit;    // [W]: bridge of worker w
    // history
    double* U_hist;
    // path
    R* path; int path_cap; int* path_len;
    // Decision trace (optional, parity tests): [trace_iters][W][kTraceInts]
    // records written by the iteration's kernels, or nullptr.
    int* trace; int trace_iters;
};

// Decision record of one worker in one iteration (fields and flags as in
// include/stp.h, stp_set_trace).
constexpr int kTraceInts = 10;
enum TraceFlag {
    kTrFwd = 1, kTrSampled = 2, kTrVirtual = 4, kTrEmit = 8, kTrRootHit = 16, kTrExtHit = 32,
    kTrInserted = 64, kTrBrCand = 128, kTrBrEmit = 256, kTrBrHit = 512, kTrWinner = 1024,
    kTrLearned = 2048, kTrLearnedT = 4096, kTrGuided = 8192
};
enum TraceField {
    kTfFlags = 0, kTfGroup = 1, kTfParent = 2, kTfExtCount = 3, kTfBrSet = 4, kTfBrIdx = 5, kTfBrCount = 6,
    kTfInserted = 7, kTfComponent = 8, kTfGoalTime = 9
};
// Record of worker w at iteration k, or nullptr when not traced.
template <typename R>
__device__ __forceinline__ int* trace_rec(const State<R>& S, int k, int w) {
    if (S.trace == nullptr || k < 0 || k >= S.trace_iters) return nullptr;
    return S.trace + ((size_t)k * S.W + w) * kTraceInts;
}

// ---------------------------------------------------------------------------
// Small helpers.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R rinf();
template <>
__device__ __forceinline__ float rinf<float>() { return __int_as_float(0x7f800000); }
template <>
__device__ __forceinline__ double rinf<double>() { return __longlong_as_double(0x7ff0000000000000LL); }

__device__ __forceinline__ void sincos_r(float x, float* s, float* c) {
    // Reduce to [-pi, pi] by whole turns (the fast intrinsic is accurate there).
    const float kTwoPi = 6.28318530717958647692f;
    const float kInvTwoPi = 0.15915494309189533577f;
    float n = rintf(x * kInvTwoPi);
    float r = fmaf(-n, kTwoPi, x);
    __sincosf(r, s, c);
}
__device__ __forceinline__ void sincos_r(double x, double* s, double* c) { sincos(x, s, c); }

__device__ __forceinline__ float rsqrt_r(float x) { return sqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return sqrt(x); }

// Philox4x32-10 (Salmon et al., SC'11), written from the published definition.
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                              uint32_t k1, uint32_t out[4]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

// ---------------------------------------------------------------------------
// Ordered-integer encodings so that atomicMin works on floating point.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ord_enc(float v) {
    int i = __float_as_int(v);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord_dec(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }
__device__ __forceinline__ long long ord_enc(double v) {
    long long i = __double_as_longlong(v);
    return i >= 0 ? i : i ^ 0x7fffffffffffffffLL;
}
__device__ __forceinline__ double ord_dec(long long i) {
    return __longlong_as_double(i >= 0 ? i : i ^ 0x7fffffffffffffffLL);
}

// ---------------------------------------------------------------------------
// TMA bulk copy + mbarrier (inline PTX).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Global -> shared bulk copy; both addresses 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ unsigned long long global_ns();

// Bounded wait for phase `parity`: gives up after limit_ns of global time (or
// the iteration backstop) and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity,
                                          unsigned long long limit_ns = kWaitLimitNs) {
    unsigned long long t0 = 0;
    for (unsigned it = 0; it < kWaitLimit; ++it) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255u) == 0) {
            const unsigned long long now = global_ns();
            if (it == 0) t0 = now;
            else if (now - t0 > limit_ns) return false;
        }
    }
    return false;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------
// Forward kinematics (standard DH; frame j+1 = frame j Rz(q_j+th0) Tz(d) Tx(a) Rx(alpha)).
// A frame is stored as columns X, Y, Z and origin o.
// ---------------------------------------------------------------------------
template <typename R>
struct Frame {
    R X[3], Y[3], Z[3], o[3];
};

template <typename R>
__device__ __forceinline__ void frame_identity(Frame<R>& F) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        F.X[i] = (i == 0) ? R(1) : R(0);
        F.Y[i] = (i == 1) ? R(1) : R(0);
        F.Z[i] = (i == 2) ? R(1) : R(0);
        F.o[i] = R(0);
    }
}

template <typename R>
__device__ __forceinline__ void frame_step(Frame<R>& F, R a, R d, R ca, R sa, R theta) {
    R s, c;
    sincos_r(theta, &s, &c);
    R u[3], w[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        u[i] = c * F.X[i] + s * F.Y[i];
        w[i] = c * F.Y[i] - s * F.X[i];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        R z = F.Z[i];
        F.X[i] = u[i];
        F.Y[i] = ca * w[i] + sa * z;
        F.Z[i] = ca * z - sa * w[i];
        F.o[i] = F.o[i] + a * u[i] + d * z;
    }
}

// Obstacle position at absolute time t from shared-memory waypoints (t,x,y,z)
// and per-segment velocities: hold before the first / after the last waypoint.
template <typename R>
__device__ __forceinline__ void obstacle_at(const R* way, const R* vel, int K, R t, R& x, R& y, R& z) {
    R tc = t > way[0] ? t : way[0];
    int k = 0;
    for (int j = 1; j < K; ++j)
        if (way[4 * j] <= tc) k = j;
    R dtk = tc - way[4 * k];
    x = way[4 * k + 1] + dtk * vel[4 * k];
    y = way[4 * k + 2] + dtk * vel[4 * k + 1];
    z = way[4 * k + 3] + dtk * vel[4 * k + 2];
}

// ---------------------------------------------------------------------------
// Planner edge batches: extension entries (2w root check, 2w+1 extension) and
// bridge entries (w), offsets scanned inside the collision kernel.
// ---------------------------------------------------------------------------
template <typename R>
__host__ __device__ inline EdgeBatch<R> ext_batch(const State<R>& S) {
    EdgeBatch<R> E;
    E.qa = S.eqa;
    E.qb = S.eqb;
    E.ta = S.eta_;
    E.tb = S.etb;
    E.qstride = kDP;
    E.cnt = S.ecnt;
    E.off = nullptr;  // offsets scanned in the kernel
    E.n_dev = nullptr;
    E.n_host = 2 * S.W;
    E.hit = S.ehit;
    E.clear = nullptr;
    E.points_done = &S.ctl->st_points;
    E.pairs_done = &S.ctl->st_pairs;
    E.err = &S.ctl->err;
    E.done = &S.ctl->done;
    return E;
}

template <typename R>
__host__ __device__ inline EdgeBatch<R> bridge_batch(const State<R>& S) {
    EdgeBatch<R> E;
    E.qa = S.bqa;
    E.qb = S.bqb;
    E.ta = S.bta;
    E.tb = S.btb;
    E.qstride = kDP;
    E.cnt = S.bcnt;
    E.off = nullptr;
    E.n_dev = nullptr;
    E.n_host = S.W;
    E.hit = S.bhit;
    E.clear = nullptr;
    E.points_done = &S.ctl->st_points;
    E.pairs_done = &S.ctl->st_pairs;
    E.err = &S.ctl->err;
    E.done = &S.ctl->done;
    return E;
}


// Batched kernels: copy problem p's Geom and State into shared memory.
template <typename R>
__device__ __forceinline__ void stage_problem(const Geom<R>* Gs, const State<R>* Ss, int p, Geom<R>& G, State<R>& S,
                                              bool with_geom = true) {
    const int* ssrc = reinterpret_cast<const int*>(Ss + p);
    int* sdst = reinterpret_cast<int*>(&S);
    if (with_geom) {
        const int* gsrc = reinterpret_cast<const int*>(Gs + p);
        int* gdst = reinterpret_cast<int*>(&G);
        for (int i = threadIdx.x; i < (int)(sizeof(Geom<R>) / sizeof(int)); i += blockDim.x) gdst[i] = gsrc[i];
    }
    for (int i = threadIdx.x; i < (int)(sizeof(State<R>) / sizeof(int)); i += blockDim.x) sdst[i] = ssrc[i];
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Launchers (explicitly instantiated in the .cu files).
// ---------------------------------------------------------------------------
template <typename R>
cudaError_t launch_validate(const Geom<R>& g, const EdgeBatch<R>& e, bool clearance, bool early_exit,
                            int grid_blocks, cudaStream_t st);
int validate_grid_blocks();

template <typename R>
cudaError_t launch_edge_counts(const Geom<R>& g, const R* qa, const R* ta, const R* qb, const R* tb, int qstride,
                               int n, double res, int* cnt, cudaStream_t st);
cudaError_t launch_scan_counts(const int* cnt, int n, long long* off, long long* block_tmp, cudaStream_t st);
cudaError_t launch_fill(void* p, long long n, int bytes, unsigned long long v, cudaStream_t st);
template <typename R>
cudaError_t launch_finish_batch(int n, const int* hit, unsigned char* verdict, R* clear, cudaStream_t st);

template <typename R>
cudaError_t launch_plan_reset(const Geom<R>& g, const State<R>& s, int max_iters, cudaStream_t st);
// Kernels of one iteration, in launch order (profiling names).
constexpr int kIterKernels = 7;
extern const char* const kIterKernelNames[kIterKernels];
// ev (optional, kIterKernels + 1 events): recorded before each kernel and after the last.
template <typename R>
cudaError_t launch_set_proposal(const Geom<R>& g, const State<R>& s, cudaStream_t st);
template <typename R>
cudaError_t launch_path_targets(const Geom<R>& g, const State<R>& s, float* out, cudaStream_t st);
template <typename R>
cudaError_t launch_iteration(const Geom<R>& g, const State<R>& s, int vgrid, cudaStream_t st,
                             cudaEvent_t* ev = nullptr);
template <typename R>
cudaError_t launch_extract_path(const State<R>& s, int dof, cudaStream_t st);

// Batched planner (problems of one precision; device arrays of Geom/State).
struct BatchShape {
    int P;               // problems
    int max_W;           // largest W
    int max_obs;         // largest obstacle count
    int validate_smem;   // dynamic shared memory of the batched collision kernel
    int nn_ctas;         // CTAs per problem for the NN and bridge scans
    int validate_ctas;   // CTAs per problem for the collision kernel
};
template <typename R>
cudaError_t launch_validate_batch(const Geom<R>* Gs, const State<R>* Ss, int P, int which, int max_obs,
                                  int ctas_per_problem, int smem_bytes, cudaStream_t st);
template <typename R>
cudaError_t launch_plan_reset_batch(const State<R>* Ss, const BatchShape& b, const int* max_iters, cudaStream_t st);
template <typename R>
cudaError_t launch_iteration_batch(const Geom<R>* Gs, const State<R>* Ss, const BatchShape& b, cudaStream_t st);
template <typename R>
cudaError_t launch_extract_path_batch(const State<R>* Ss, const BatchShape& b, cudaStream_t st);

}  // namespace stp
