// Collision-kernel launches: the stand-alone edge batch (stp_check_edges),
// the planner's per-step launches and the batched form, plus the flat-batch
// helpers (check counts, prefix sums, fills). The device code of a check
// point and of a batch lives in stp_validate_body.cuh.
#include "stp_validate_body.cuh"

namespace stp {

template <typename R, bool ARM, int MO, bool CLEAR, bool EARLY>
__global__ void __launch_bounds__(256, (sizeof(R) == 4 && MO <= 16) ? 2 : 1) k_validate(Geom<R> G, EdgeBatch<R> E) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    validate_body<R, ARM, MO, CLEAR, EARLY>(G, E, smem_raw, blockIdx.x, gridDim.x);
}

// Batched planner form: problem blockIdx.y; its geometry and state are staged
// in shared memory, its extension (which = 0) or bridge (which = 1) edge
// entries are validated; arm vs point robot is chosen per problem.
template <typename R, int MO>
__global__ void __launch_bounds__(256, (sizeof(R) == 4 && MO <= 16) ? 2 : 1)
    k_validate_batch(const Geom<R>* __restrict__ Gs, const State<R>* __restrict__ Ss, int which) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Geom<R> G;
    __shared__ State<R> S;
    stage_problem(Gs, Ss, blockIdx.y, G, S);
    EdgeBatch<R> E = which == 0 ? ext_batch(S) : bridge_batch(S);
    E.phase = which >= 1 ? which : 0;   // which 1: coarse bridge pass, 2: remaining bridge points
    if (G.arm) validate_body<R, true, MO, false, true>(G, E, smem_raw, blockIdx.x, gridDim.x);
    else validate_body<R, false, MO, false, true>(G, E, smem_raw, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
int validate_grid_blocks() {
    static std::mutex mu;
    static int sms[kMaxDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 1;
    std::lock_guard<std::mutex> lock(mu);
    if (sms[dev] == 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        sms[dev] = n > 0 ? n : 1;
    }
    return sms[dev];
}

template <typename R, bool ARM, int MO, bool CLEAR, bool EARLY>
static cudaError_t launch_v(const Geom<R>& g, const EdgeBatch<R>& e, int grid_blocks, cudaStream_t st) {
    auto kern = k_validate<R, ARM, MO, CLEAR, EARLY>;
    static SmemAttr attr;
    static int blocks_per_sm[kMaxDevices] = {};  // resident CTAs at the configured size
    int smem = (int)g.blob_bytes + (e.off ? (int)(sizeof(long long) * (kWin + 1))
                                          : (int)(sizeof(int) * (e.n_host + 1)));
    bool raised = false;
    cudaError_t err = ensure_smem((const void*)kern, attr, smem, &raised);
    if (err != cudaSuccess) return err;
    int dev = 0;
    err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (raised || blocks_per_sm[dev] == 0) {
        int b = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 256, smem);
        if (err != cudaSuccess) return err;
        blocks_per_sm[dev] = b < 1 ? 1 : b;
    }
    int grid = grid_blocks > 0 ? grid_blocks : validate_grid_blocks() * blocks_per_sm[dev];
    kern<<<grid, 256, smem, st>>>(g, e);
    return cudaGetLastError();
}

// Obstacle chunk per pass: FP32 keeps at most 16 obstacles in registers
// (128 registers, two CTAs per SM; more obstacles take more passes, each
// repeating the forward kinematics), FP64 up to 32.
template <typename R, bool ARM, bool CLEAR, bool EARLY>
static cudaError_t launch_mo(const Geom<R>& g, const EdgeBatch<R>& e, int grid_blocks, cudaStream_t st) {
    if (CLEAR) return launch_v<R, ARM, 16, CLEAR, EARLY>(g, e, grid_blocks, st);
    if (g.M <= 8) return launch_v<R, ARM, 8, CLEAR, EARLY>(g, e, grid_blocks, st);
    if constexpr (sizeof(R) == 4) {
        return launch_v<R, ARM, 16, CLEAR, EARLY>(g, e, grid_blocks, st);
    } else {
        if (g.M <= 16) return launch_v<R, ARM, 16, CLEAR, EARLY>(g, e, grid_blocks, st);
        return launch_v<R, ARM, 32, CLEAR, EARLY>(g, e, grid_blocks, st);
    }
}

// ---------------------------------------------------------------------------
// Closed-form (continuous) validation of point-robot edges, one lane per
// edge. Between consecutive breakpoints (the edge's end times and each
// obstacle waypoint time inside them) a robot sphere and an obstacle both
// move linearly, so their difference runs along the segment from d(t0) to
// d(t1) and its smallest norm is the distance from the origin to that segment.
// A pair collides iff that squared minimum < (r + r_o)^2; the edge stays in
// the convex configuration box iff both ends do.
// ---------------------------------------------------------------------------
template <typename R, bool CLEAR>
__global__ void __launch_bounds__(256) k_validate_cont(Geom<R> G, EdgeBatch<R> E) {
    const int n = E.n_dev ? *E.n_dev : E.n_host;
    if (n <= 0 || (E.done && *E.done)) return;
    const R* sph = G.blob;
    const R* way = G.blob + G.off_way;
    const R* vel = G.blob + G.off_vel;
    const R* rad = G.blob + G.off_rad;
    unsigned long long done = 0, pairs_total = 0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        if (E.cnt[e] <= 0) continue;
        const R* qa = E.qa + (size_t)e * E.qstride;
        const R* qb = E.qb + (size_t)e * E.qstride;
        const R ta = E.ta[e], tb = E.tb[e];
        bool hit = false;
        for (int j = 0; j < G.dof; ++j)
            hit = hit || qa[j] < G.qlo[j] || qa[j] > G.qhi[j] || qb[j] < G.qlo[j] || qb[j] > G.qhi[j];
        const R pa[3] = {qa[0], qa[1], G.dof > 2 ? qa[2] : R(0)};
        const R pb[3] = {qb[0], qb[1], G.dof > 2 ? qb[2] : R(0)};
        R clr = rinf<R>();
        for (int m = 0; m < G.M; ++m) {
            const R* W = way + 4 * G.K * m;
            const R* V = vel + 4 * G.K * m;
            const R ro = rad[m];
            R t0 = ta;
            for (int k = 0; k <= G.K; ++k) {
                // next breakpoint: waypoint k if inside (ta, tb), the end at k == K
                R t1;
                if (k < G.K) {
                    t1 = W[4 * k];
                    if (!(t1 > ta && t1 < tb)) continue;
                } else {
                    t1 = tb;
                }
                const R f0 = tb > ta ? (t0 - ta) / (tb - ta) : R(0);
                const R f1 = tb > ta ? (t1 - ta) / (tb - ta) : R(0);
                R o0[3], o1[3];
                obstacle_at(W, V, G.K, t0, o0[0], o0[1], o0[2]);
                obstacle_at(W, V, G.K, t1, o1[0], o1[1], o1[2]);
                for (int sp = 0; sp < G.S; ++sp) {
                    R d0[3], w[3];
                    for (int i = 0; i < 3; ++i) {
                        const R c0 = (pa[i] + f0 * (pb[i] - pa[i])) + sph[4 * sp + i];
                        const R c1 = (pa[i] + f1 * (pb[i] - pa[i])) + sph[4 * sp + i];
                        d0[i] = c0 - o0[i];
                        w[i] = (c1 - o1[i]) - d0[i];
                    }
                    const R a = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
                    const R b = d0[0] * w[0] + d0[1] * w[1] + d0[2] * w[2];
                    R u = a > R(0) ? -b / a : R(0);
                    u = u < R(0) ? R(0) : (u > R(1) ? R(1) : u);
                    R d2 = R(0);
                    for (int i = 0; i < 3; ++i) {
                        const R x = d0[i] + u * w[i];
                        d2 += x * x;
                    }
                    const R rr = sph[4 * sp + 3] + ro;
                    hit = hit || (d2 < rr * rr);
                    if (CLEAR) {
                        const R cl = rsqrt_r(d2) - rr;
                        clr = cl < clr ? cl : clr;
                    }
                }
                pairs_total += (unsigned long long)G.S;
                t0 = t1;
            }
        }
        E.hit[e] = hit ? 1 : 0;
        if (CLEAR) atomic_min_r<R>(E.clear + e, clr);  // order-encoded like the discrete path
        ++done;
    }
    const int lane = threadIdx.x & 31;
    if (E.points_done) {
        for (int o = 16; o > 0; o >>= 1) done += __shfl_xor_sync(0xffffffffu, done, o);
        if (lane == 0 && done) atomicAdd(E.points_done, done);
    }
    if (E.pairs_done) {
        for (int o = 16; o > 0; o >>= 1) pairs_total += __shfl_xor_sync(0xffffffffu, pairs_total, o);
        if (lane == 0 && pairs_total) atomicAdd(E.pairs_done, pairs_total);
    }
}

template <typename R>
cudaError_t launch_validate(const Geom<R>& g, const EdgeBatch<R>& e, bool clearance, bool early_exit,
                            int grid_blocks, cudaStream_t st) {
    if (g.continuous) {
        const int blocks = grid_blocks > 0 ? grid_blocks : validate_grid_blocks() * 2;
        if (clearance) k_validate_cont<R, true><<<blocks, 256, 0, st>>>(g, e);
        else k_validate_cont<R, false><<<blocks, 256, 0, st>>>(g, e);
        return cudaGetLastError();
    }
    if (g.arm) {
        if (clearance) return launch_mo<R, true, true, false>(g, e, grid_blocks, st);
        if (early_exit) return launch_mo<R, true, false, true>(g, e, grid_blocks, st);
        return launch_mo<R, true, false, false>(g, e, grid_blocks, st);
    }
    if (clearance) return launch_mo<R, false, true, false>(g, e, grid_blocks, st);
    if (early_exit) return launch_mo<R, false, false, true>(g, e, grid_blocks, st);
    return launch_mo<R, false, false, false>(g, e, grid_blocks, st);
}

template <typename R, int MO>
static cudaError_t launch_vb(const Geom<R>* Gs, const State<R>* Ss, int P, int which, int ctas_per_problem,
                             int smem_bytes, cudaStream_t st) {
    auto kern = k_validate_batch<R, MO>;
    static SmemAttr attr;
    cudaError_t err = ensure_smem((const void*)kern, attr, smem_bytes);
    if (err != cudaSuccess) return err;
    if (P <= 0) return cudaSuccess;  // configuration only
    kern<<<dim3(ctas_per_problem, P), 256, smem_bytes, st>>>(Gs, Ss, which);
    return cudaGetLastError();
}

// P <= 0 only sets the kernel's shared-memory attribute (nothing is launched).
template <typename R>
cudaError_t launch_validate_batch(const Geom<R>* Gs, const State<R>* Ss, int P, int which, int max_obs,
                                  int ctas_per_problem, int smem_bytes, cudaStream_t st) {
    if (max_obs <= 8) return launch_vb<R, 8>(Gs, Ss, P, which, ctas_per_problem, smem_bytes, st);
    return launch_vb<R, 16>(Gs, Ss, P, which, ctas_per_problem, smem_bytes, st);
}
template cudaError_t launch_validate_batch<float>(const Geom<float>*, const State<float>*, int, int, int, int, int,
                                                  cudaStream_t);

// Check-point counts, c = max(1, ceil(max(D, v_max |dt|) / res - 1e-3)),
// evaluated in double from the stored endpoints.
template <typename R>
__global__ void k_edge_counts(double vmax, int dof, const R* qa, const R* ta, const R* qb, const R* tb, int qstride,
                              int n, double res, int* cnt) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double s2 = 0.0;
    for (int i = 0; i < dof; ++i) {
        double dd = (double)qb[(size_t)e * qstride + i] - (double)qa[(size_t)e * qstride + i];
        s2 = __dadd_rn(s2, __dmul_rn(dd, dd));
    }
    double D = sqrt(s2);
    double L = fmax(D, __dmul_rn(vmax, fabs((double)tb[e] - (double)ta[e])));
    double c = ceil(L / res - 1e-3);
    cnt[e] = c < 1.0 ? 1 : (int)c;
}

template <typename R>
cudaError_t launch_edge_counts(const Geom<R>& g, const R* qa, const R* ta, const R* qb, const R* tb, int qstride,
                               int n, double res, int* cnt, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_edge_counts<R><<<(n + 255) / 256, 256, 0, st>>>(g.vmax_d, g.dof, qa, ta, qb, tb, qstride, n, res, cnt);
    return cudaGetLastError();
}

// Exclusive prefix sum of counts into off[0..n] (off[n] = total); three phases.
constexpr int kScanBlock = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanBlock * kScanPer;

__device__ __forceinline__ long long block_exclusive_scan(long long v, long long* sh, long long* total) {
    // Warp scan then scan of warp totals.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        long long w = lane < nw ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) sh[lane] = w;
    }
    __syncthreads();
    long long before = (warp > 0 ? sh[warp - 1] : 0) + x - v;
    if (total) *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void k_scan_tiles(const int* cnt, int n, long long* off, long long* tile_tot) {
    __shared__ long long sh[32];
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanPer;
    long long v[kScanPer];
    long long sum = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        v[i] = (base + i < n) ? cnt[base + i] : 0;
        sum += v[i];
    }
    long long tot;
    long long pre = block_exclusive_scan(sum, sh, &tot);
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        if (base + i < n) off[base + i] = pre;
        pre += v[i];
    }
    if (threadIdx.x == 0) tile_tot[blockIdx.x] = tot;
}

__global__ void k_scan_tops(long long* tile_tot, int ntiles, long long* off, int n) {
    __shared__ long long sh[32];
    long long carry = 0;
    for (int b0 = 0; b0 < ntiles; b0 += blockDim.x) {
        int b = b0 + threadIdx.x;
        long long v = b < ntiles ? tile_tot[b] : 0;
        long long tot;
        long long pre = block_exclusive_scan(v, sh, &tot);
        if (b < ntiles) tile_tot[b] = carry + pre;
        carry += tot;
    }
    if (threadIdx.x == 0) off[n] = carry;
}

__global__ void k_scan_add(long long* off, int n, const long long* tile_tot) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) off[i] += tile_tot[i / kScanTile];
}

cudaError_t launch_scan_counts(const int* cnt, int n, long long* off, long long* tile_tmp, cudaStream_t st) {
    if (n <= 0) {
        return cudaMemsetAsync(off, 0, sizeof(long long), st);
    }
    int ntiles = (n + kScanTile - 1) / kScanTile;
    k_scan_tiles<<<ntiles, kScanBlock, 0, st>>>(cnt, n, off, tile_tmp);
    k_scan_tops<<<1, kScanBlock, 0, st>>>(tile_tmp, ntiles, off, n);
    k_scan_add<<<(n + 255) / 256, 256, 0, st>>>(off, n, tile_tmp);
    return cudaGetLastError();
}

// Small fills and conversions used by the batch entry point.
__global__ void k_fill_u32(unsigned* p, long long n, unsigned v) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}
__global__ void k_fill_u64(unsigned long long* p, long long n, unsigned long long v) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}
cudaError_t launch_fill(void* p, long long n, int bytes, unsigned long long v, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int grid = (int)((n + 255) / 256);
    if (bytes == 4) k_fill_u32<<<grid, 256, 0, st>>>((unsigned*)p, n, (unsigned)v);
    else k_fill_u64<<<grid, 256, 0, st>>>((unsigned long long*)p, n, v);
    return cudaGetLastError();
}

template <typename R>
__global__ void k_finish_batch(int n, const int* hit, unsigned char* verdict, R* clear) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    verdict[e] = hit[e] ? 0 : 1;
    if (clear) clear[e] = ord_dec(*reinterpret_cast<const decltype(ord_enc(R(0)))*>(clear + e));
}
template <typename R>
cudaError_t launch_finish_batch(int n, const int* hit, unsigned char* verdict, R* clear, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_finish_batch<R><<<(n + 255) / 256, 256, 0, st>>>(n, hit, verdict, clear);
    return cudaGetLastError();
}
template cudaError_t launch_finish_batch<float>(int, const int*, unsigned char*, float*, cudaStream_t);
template cudaError_t launch_finish_batch<double>(int, const int*, unsigned char*, double*, cudaStream_t);

template cudaError_t launch_validate<float>(const Geom<float>&, const EdgeBatch<float>&, bool, bool, int,
                                            cudaStream_t);
template cudaError_t launch_validate<double>(const Geom<double>&, const EdgeBatch<double>&, bool, bool, int,
                                             cudaStream_t);
template cudaError_t launch_edge_counts<float>(const Geom<float>&, const float*, const float*, const float*,
                                               const float*, int, int, double, int*, cudaStream_t);
template cudaError_t launch_edge_counts<double>(const Geom<double>&, const double*, const double*, const double*,
                                                const double*, int, int, double, int*, cudaStream_t);

}  // namespace stp
