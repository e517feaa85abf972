// C ABI of the ST-pRRTC batched space-time Extend library (declarations and
// contracts in include/stp.h). Host code: validation, one device arena per
// problem, the geometry blob, goal-time grid checks at creation, and CUDA
// graphs that hold a fixed number of planner iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "stp.h"
#include "stp_internal.cuh"
#include "stp_persist.cuh"

using namespace stp;

namespace {

const double kInfD = std::numeric_limits<double>::infinity();

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Device resources kept for reuse across problems: memory blocks (by device
// and size), non-blocking streams (by device) and instantiated iteration
// graphs (by device). Creating and freeing many short-lived problems then
// costs no cudaMalloc/cudaFree (and none of the device synchronisation of
// cudaFree), and a new problem's captured iteration graph updates an idle
// executable graph of the same topology (cudaGraphExecUpdate: new kernel
// parameters) instead of being instantiated. Resources are handed out only
// when idle: stp_free synchronises the problem's streams first.
// stp_release_cached() returns everything to the driver.
struct DevCache {
    std::mutex mu;
    struct Block {
        int dev;
        void* ptr;
    };
    std::multimap<size_t, Block> blocks;
    size_t cached = 0;
    std::vector<std::pair<int, cudaStream_t>> streams;
    std::vector<std::pair<int, cudaGraphExec_t>> graphs;
};
constexpr size_t kCacheLimit = size_t(4) << 30;  // bytes of idle blocks kept
constexpr size_t kGraphCache = 8;                // idle executable graphs kept

DevCache& dev_cache() {
    // Never destroyed: no CUDA call may run during static destruction.
    static DevCache* c = new DevCache();
    return *c;
}

int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

// A block of at least `bytes` (at most twice that plus 1 MiB, so small
// requests do not pin large blocks); *got receives its size.
cudaError_t cache_alloc(void** ptr, size_t bytes, size_t* got) {
    bytes = align_up(std::max<size_t>(bytes, 256), 256);
    const int dev = current_device();
    {
        DevCache& c = dev_cache();
        std::lock_guard<std::mutex> g(c.mu);
        for (auto it = c.blocks.lower_bound(bytes); it != c.blocks.end() && it->first <= 2 * bytes + (1 << 20);
             ++it) {
            if (it->second.dev != dev) continue;
            *ptr = it->second.ptr;
            *got = it->first;
            c.cached -= it->first;
            c.blocks.erase(it);
            return cudaSuccess;
        }
    }
    *got = bytes;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e == cudaErrorMemoryAllocation) {
        // Out of memory: hand this device's idle blocks back to the driver and retry once.
        (void)cudaGetLastError();
        std::vector<void*> idle;
        {
            DevCache& c = dev_cache();
            std::lock_guard<std::mutex> g(c.mu);
            for (auto it = c.blocks.begin(); it != c.blocks.end();) {
                if (it->second.dev == dev) {
                    idle.push_back(it->second.ptr);
                    c.cached -= it->first;
                    it = c.blocks.erase(it);
                } else {
                    ++it;
                }
            }
        }
        if (!idle.empty()) {
            for (void* q : idle) cudaFree(q);
            e = cudaMalloc(ptr, bytes);
        }
    }
    return e;
}

void cache_release(void* ptr, size_t bytes) {
    if (!ptr) return;
    {
        DevCache& c = dev_cache();
        std::lock_guard<std::mutex> g(c.mu);
        if (c.cached + bytes <= kCacheLimit) {
            c.blocks.emplace(bytes, DevCache::Block{current_device(), ptr});
            c.cached += bytes;
            return;
        }
    }
    cudaFree(ptr);
}

cudaError_t cache_stream(cudaStream_t* st) {
    const int dev = current_device();
    {
        DevCache& c = dev_cache();
        std::lock_guard<std::mutex> g(c.mu);
        for (size_t i = 0; i < c.streams.size(); ++i) {
            if (c.streams[i].first != dev) continue;
            *st = c.streams[i].second;
            c.streams.erase(c.streams.begin() + (long)i);
            return cudaSuccess;
        }
    }
    return cudaStreamCreateWithFlags(st, cudaStreamNonBlocking);
}

void cache_stream_release(cudaStream_t st) {
    if (!st) return;
    DevCache& c = dev_cache();
    std::lock_guard<std::mutex> g(c.mu);
    c.streams.emplace_back(current_device(), st);
}

// An executable graph for the captured graph g: the most recently released
// idle one of this device updated to g, else a new instantiation. An update
// that fails (another topology) leaves nothing behind: that executable graph
// is destroyed and the error state cleared.
cudaError_t cache_graph_exec(cudaGraph_t g, cudaGraphExec_t* out) {
    const int dev = current_device();
    cudaGraphExec_t ex = nullptr;
    {
        DevCache& c = dev_cache();
        std::lock_guard<std::mutex> lock(c.mu);
        for (size_t i = c.graphs.size(); i-- > 0;) {
            if (c.graphs[i].first != dev) continue;
            ex = c.graphs[i].second;
            c.graphs.erase(c.graphs.begin() + (long)i);
            break;
        }
    }
    if (ex) {
        cudaGraphExecUpdateResultInfo info{};
        if (cudaGraphExecUpdate(ex, g, &info) == cudaSuccess) {
            *out = ex;
            return cudaSuccess;
        }
        (void)cudaGetLastError();
        cudaGraphExecDestroy(ex);
    }
    return cudaGraphInstantiate(out, g, 0);
}

// Keep an idle executable graph (its launches finished) for cache_graph_exec.
void cache_graph_release(cudaGraphExec_t ex) {
    if (!ex) return;
    {
        DevCache& c = dev_cache();
        std::lock_guard<std::mutex> g(c.mu);
        if (c.graphs.size() < kGraphCache) {
            c.graphs.emplace_back(current_device(), ex);
            return;
        }
    }
    cudaGraphExecDestroy(ex);
}

// Carves aligned sub-buffers out of one device allocation.
struct Carver {
    size_t off = 0;
    char* base = nullptr;
    template <typename T>
    T* take(size_t count) {
        off = align_up(off, 256);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

}  // namespace

struct stp_problem {
    int precision = 0;
    int dof = 0, arm = 0, S = 0, M = 0, K = 0;
    stp_params prm{};
    std::vector<double> qs, qg, qlo, qhi, dh, sph, obs_r, way;
    double vmax = 1.0;
    double Lg = 0.0;
    long long kmin = 0, kmax = -1, kend = 0;
    int nk = 0;
    int start_free = 0;
    int cap_f = 0, cap_s = 0, cap_trees = 0, max_pieces = 0, path_cap = 0;
    char* d_arena = nullptr;
    size_t arena_bytes = 0;
    size_t arena_block = 0;   // size of the (possibly reused) block holding the arena
    Geom<float> gf{};
    Geom<double> gd{};
    State<float> sf{};
    State<double> sd{};
    Ctl* d_ctl = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t graph_stream = nullptr;
    int graph_iters = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;
    cudaEvent_t ev_step0 = nullptr, ev_step1 = nullptr;  // every GPU operation of a stp_plan call
    // batch scratch for stp_check_edges
    char* d_scratch = nullptr;
    size_t scratch_bytes = 0;
    unsigned long long* d_counters = nullptr;  // [2]: points, pairs of stp_check_edges
    size_t counters_block = 0;
    std::string last_error;
    bool planned = false;
    bool has_proposal = false;  // learned branch table set by stp_set_proposal
    std::vector<int> self_pairs;  // self-collision pairs a * 64 + b (device sphere order)
    // persistent launch: device copies of the problem's Geom / State (refreshed
    // before each launch), its iteration budget and the launch scratch
    void* d_pgeom = nullptr;
    void* d_pstate = nullptr;
    int* d_pmax_iters = nullptr;
    PersistScratch pscratch{};
    size_t pscratch_bytes = 0;
    int persist_grid = 0, persist_smem = 0, persist_dq = 0;
    // decision trace (stp_set_trace): [trace_iters][W][kTraceInts]
    int* d_trace = nullptr;
    int trace_iters = 0;
    int* graph_trace = nullptr;  // trace pointer the captured graph was built with
    // profiling
    int profiling = 0;
    std::vector<cudaEvent_t> prof_ev;
    double prof_ms[kIterKernels] = {};
    long long prof_launches[kIterKernels] = {};
};

namespace {

// Last failure of any call (also of calls that have no problem handle yet).
thread_local std::string g_last_error;

// A non-sticky error left by an earlier runtime call of this thread (ours or
// the caller's) must not be reported by our own launch checks.
void clear_stale_error() { (void)cudaGetLastError(); }

stp_status cuda_fail(stp_problem* p, cudaError_t e, const char* where) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
    if (p) p->last_error = buf;
    g_last_error = buf;
    return STP_ERR_CUDA;
}

#define STP_CUDA(p, call)                                   \
    do {                                                    \
        cudaError_t _e = (call);                            \
        if (_e != cudaSuccess) return cuda_fail(p, _e, #call); \
    } while (0)

bool finite_all(const double* a, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

double host_dist(const double* a, const double* b, int d) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        double e = b[j] - a[j];
        s += e * e;
    }
    return std::sqrt(s);
}

template <typename R>
void fill_geom(stp_problem* p, Geom<R>& g, const R* blob, unsigned blob_bytes, int off_way, int off_vel,
               int off_rad, int off_tim, int off_self, const std::vector<int>& link_start) {
    std::memset(&g, 0, sizeof(g));
    g.dof = p->dof;
    g.arm = p->arm;
    g.S = p->S;
    g.M = p->M;
    g.K = p->K;
    g.DP = kDP;
    for (int j = 0; j < kMaxDof + 2; ++j) g.link_start[j] = j < (int)link_start.size() ? link_start[j] : p->S;
    for (int j = 0; j < p->dof; ++j) {
        if (p->arm) {
            g.a[j] = (R)p->dh[4 * j];
            g.ca[j] = (R)std::cos(p->dh[4 * j + 1]);
            g.sa[j] = (R)std::sin(p->dh[4 * j + 1]);
            g.d[j] = (R)p->dh[4 * j + 2];
            g.th0[j] = (R)p->dh[4 * j + 3];
        }
        g.qlo[j] = (R)p->qlo[j];
        g.qhi[j] = (R)p->qhi[j];
    }
    g.vmax = (R)p->vmax;
    g.vmax_d = p->vmax;
    // Reference point for the pair tests: the arm base, or the centre of a
    // point robot's configuration box.
    for (int i = 0; i < 3; ++i) g.ref[i] = R(0);
    if (!p->arm)
        for (int i = 0; i < 3 && i < p->dof; ++i) g.ref[i] = (R)(0.5 * (p->qlo[i] + p->qhi[i]));
    g.continuous = p->prm.continuous;
    g.uniform_ro = 1;
    for (int m = 1; m < p->M; ++m)
        if (p->obs_r[m] != p->obs_r[0]) g.uniform_ro = 0;
    g.ro_uni = p->M > 0 ? (R)p->obs_r[0] : R(0);
    g.blob = blob;
    g.blob_bytes = blob_bytes;
    g.off_way = off_way;
    g.off_vel = off_vel;
    g.off_rad = off_rad;
    g.off_tim = off_tim;
    g.off_self = off_self;
    g.n_self = (int)p->self_pairs.size();
}

// Self-collision pairs in the device sphere order (reading: spheres on frames
// at least two apart, excluding pairs that already overlap at q = 0), encoded
// a * 64 + b with a < b. Zero-configuration FK in FP64, standard DH.
void compute_self_pairs(stp_problem* p, const std::vector<int>& order) {
    p->self_pairs.clear();
    if (!p->prm.self_collision || !p->arm) return;
    struct F3 {
        double X[3], Y[3], Z[3], o[3];
    };
    std::vector<F3> fr(1);
    for (int i = 0; i < 3; ++i) {
        fr[0].X[i] = i == 0;
        fr[0].Y[i] = i == 1;
        fr[0].Z[i] = i == 2;
        fr[0].o[i] = 0.0;
    }
    for (int j = 0; j < p->dof; ++j) {
        const double a = p->dh[4 * j], al = p->dh[4 * j + 1], d = p->dh[4 * j + 2], th = p->dh[4 * j + 3];
        const double c = std::cos(th), sn = std::sin(th), ca = std::cos(al), sa = std::sin(al);
        F3 f = fr.back(), g;
        for (int i = 0; i < 3; ++i) {
            const double u = c * f.X[i] + sn * f.Y[i], w = c * f.Y[i] - sn * f.X[i], z = f.Z[i];
            g.X[i] = u;
            g.Y[i] = ca * w + sa * z;
            g.Z[i] = ca * z - sa * w;
            g.o[i] = f.o[i] + a * u + d * z;
        }
        fr.push_back(g);
    }
    const int S = p->S;
    std::vector<double> cs(3 * (size_t)S);
    std::vector<int> link(S);
    for (int k = 0; k < S; ++k) {
        const double* sp = &p->sph[5 * order[k]];
        const F3& f = fr[(int)sp[0]];
        link[k] = (int)sp[0];
        for (int i = 0; i < 3; ++i) cs[3 * k + i] = f.o[i] + sp[1] * f.X[i] + sp[2] * f.Y[i] + sp[3] * f.Z[i];
    }
    for (int a = 0; a < S; ++a)
        for (int b = a + 1; b < S; ++b) {
            if (std::abs(link[a] - link[b]) < 2) continue;
            double d2 = 0.0;
            for (int i = 0; i < 3; ++i) d2 += (cs[3 * a + i] - cs[3 * b + i]) * (cs[3 * a + i] - cs[3 * b + i]);
            const double rr = p->sph[5 * order[a] + 4] + p->sph[5 * order[b] + 4];
            if (d2 < rr * rr) continue;
            p->self_pairs.push_back(a * 64 + b);
        }
}

// Sizes and layout of the geometry blob in R units; returns bytes.
template <typename R>
size_t blob_layout(const stp_problem* p, int* off_way, int* off_vel, int* off_rad, int* off_tim, int* off_self) {
    size_t n = 4 * (size_t)p->S;
    *off_way = (int)n;
    n += 4 * (size_t)p->M * p->K;
    *off_vel = (int)n;
    n += 4 * (size_t)p->M * p->K;
    *off_rad = (int)n;
    n += align_up((size_t)p->M, 4);
    *off_tim = (int)n;
    n += (size_t)kMaxWay * p->M;
    *off_self = (int)n;
    n += p->self_pairs.size();
    if (n == 0) n = 4;
    return align_up(n * sizeof(R), 16);
}

template <typename R>
std::vector<R> blob_host(const stp_problem* p, const std::vector<int>& order, size_t bytes, int off_way,
                         int off_vel, int off_rad, int off_tim, int off_self) {
    std::vector<R> b(bytes / sizeof(R), R(0));
    for (int s = 0; s < p->S; ++s) {
        const double* sp = &p->sph[5 * order[s]];
        for (int i = 0; i < 4; ++i) b[4 * s + i] = (R)sp[1 + i];
    }
    for (int m = 0; m < p->M; ++m) {
        for (int k = 0; k < p->K; ++k) {
            const double* w = &p->way[((size_t)m * p->K + k) * 4];
            for (int i = 0; i < 4; ++i) b[off_way + ((size_t)m * p->K + k) * 4 + i] = (R)w[i];
            double v[3] = {0, 0, 0};
            if (k + 1 < p->K) {
                const double* w1 = w + 4;
                double dt = w1[0] - w[0];
                for (int i = 0; i < 3; ++i) v[i] = (w1[1 + i] - w[1 + i]) / dt;
            }
            for (int i = 0; i < 3; ++i) b[off_vel + ((size_t)m * p->K + k) * 4 + i] = (R)v[i];
        }
        b[off_rad + m] = (R)p->obs_r[m];
        for (int k = 1; k <= kMaxWay; ++k)
            b[off_tim + (size_t)m * kMaxWay + k - 1] =
                k < p->K ? (R)p->way[((size_t)m * p->K + k) * 4] : std::numeric_limits<R>::infinity();
    }
    for (size_t i = 0; i < p->self_pairs.size(); ++i) b[off_self + i] = (R)p->self_pairs[i];
    return b;
}

template <typename R>
State<R>& state_of(stp_problem* p);
template <>
State<float>& state_of<float>(stp_problem* p) { return p->sf; }
template <>
State<double>& state_of<double>(stp_problem* p) { return p->sd; }
template <typename R>
Geom<R>& geom_of(stp_problem* p);
template <>
Geom<float>& geom_of<float>(stp_problem* p) { return p->gf; }
template <>
Geom<double>& geom_of<double>(stp_problem* p) { return p->gd; }

// Lays out (base == nullptr: sizes only) every device buffer of a problem.
template <typename R>
size_t layout_state(stp_problem* p, char* base, R** blob_out, size_t blob_bytes, unsigned char** gfree,
                    Ctl** ctl, R** qdev, R** tdev, int** cnt, long long** off, int** hit) {
    Carver cv;
    cv.base = base;
    const int W = p->prm.ext_per_iter, N = p->prm.n_roots;
    State<R> s;
    std::memset(&s, 0, sizeof(s));
    *ctl = cv.take<Ctl>(1);
    *blob_out = reinterpret_cast<R*>(cv.take<char>(blob_bytes));
    *gfree = cv.take<unsigned char>(std::max(p->nk, 1) + 1);
    // goal grid / start check scratch
    const int ng = p->nk + 1;
    *qdev = cv.take<R>(kDP);
    *tdev = cv.take<R>(ng);
    *cnt = cv.take<int>(ng);
    *off = cv.take<long long>(ng + 1);
    *hit = cv.take<int>(ng);
    s.ctl = *ctl;
    s.fx = cv.take<R>((size_t)p->cap_f * kDP);
    s.fpar = cv.take<int>(p->cap_f);
    s.fcost = cv.take<R>(p->cap_f);
    s.fiter = cv.take<int>(p->cap_f);
    const size_t nb = (size_t)N * p->cap_s;
    s.bx = cv.take<R>(nb * kDP);
    s.bpar = cv.take<int>(nb);
    s.bcost = cv.take<R>(nb);
    s.btroot = cv.take<R>(nb);
    s.btree = cv.take<int>(nb);
    s.biter = cv.take<int>(nb);
    s.tree_group = cv.take<int>(p->cap_trees);
    s.tree_T = cv.take<double>(p->cap_trees);
    const int nwin = std::max(p->nk, 1);
    s.win_lo = cv.take<double>(nwin);
    s.win_hi = cv.take<double>(nwin);
    s.pc_lo = cv.take<double>(p->max_pieces);
    s.pc_hi = cv.take<double>(p->max_pieces);
    s.pc_group = cv.take<int>(p->max_pieces);
    s.gfree = *gfree;
    s.w_status = cv.take<int>(W);
    s.w_set = cv.take<int>(W);
    s.w_xr = cv.take<R>((size_t)W * kDP);
    s.w_T = cv.take<R>(W);
    s.w_parent = cv.take<int>(W);
    s.w_key = cv.take<R>(W);
    s.w_xnew = cv.take<R>((size_t)W * kDP);
    s.w_edge = cv.take<int>(W);
    s.w_root_edge = cv.take<int>(W);
    s.w_ins = cv.take<int>(W);
    s.w_bedge = cv.take<int>(W);
    s.w_xn = cv.take<R>((size_t)W * kDP);
    s.w_nnkey = cv.take<unsigned long long>(W);
    s.qlist = cv.take<int>((size_t)(N + 1) * W);
    s.tile_cnt = cv.take<int>((size_t)(N + 1) * kMaxQTiles);
    // Per-tile partials serve the FP64 scans only (FP32 merges keys atomically).
    const size_t npart = sizeof(R) == 8 ? (size_t)W * kMaxTiles : 0;
    s.part_k1 = cv.take<R>(npart);
    s.part_k2 = cv.take<R>(npart);
    s.part_idx = cv.take<int>(npart);
    s.bq_list = cv.take<int>((size_t)2 * W);
    s.bq_count = cv.take<int>(2);
    s.btile_cnt = cv.take<int>((size_t)2 * kMaxQTiles);
    s.bkey = cv.take<unsigned long long>((size_t)2 * W);
    s.b_set = cv.take<int>(W);
    s.b_idx = cv.take<int>(W);
    s.b_k1 = cv.take<R>(W);
    s.b_k2 = cv.take<R>(W);
    s.b_U = cv.take<R>(W);
    s.b_C = cv.take<R>(W);
    s.eqa = cv.take<R>((size_t)2 * W * kDP);
    s.eqb = cv.take<R>((size_t)2 * W * kDP);
    s.eta_ = cv.take<R>((size_t)2 * W);
    s.etb = cv.take<R>((size_t)2 * W);
    s.ecnt = cv.take<int>((size_t)2 * W);
    s.ehit = cv.take<int>((size_t)2 * W);
    s.bqa = cv.take<R>((size_t)W * kDP);
    s.bqb = cv.take<R>((size_t)W * kDP);
    s.bta = cv.take<R>(W);
    s.btb = cv.take<R>(W);
    s.bcnt = cv.take<int>(W);
    s.bhit = cv.take<int>(W);
    s.U_hist = cv.take<double>(std::max(p->prm.max_iters, 1));
    s.path = cv.take<R>((size_t)p->path_cap * kDP);
    s.path_len = cv.take<int>(1);
    s.prop = cv.take<R>(kPropSize);
    s.prop_y = cv.take<float>(kPropY);
    s.tgt = cv.take<float>(STP_MLP_NTGT + 1);
    // persistent launch (one team)
    void* pg = cv.take<Geom<R>>(1);
    void* ps = cv.take<State<R>>(1);
    int* pmi = cv.take<int>(1);
    char* pscr = cv.take<char>(persist_scratch_bytes(1));
    if (base) {
        p->d_pgeom = pg;
        p->d_pstate = ps;
        p->d_pmax_iters = pmi;
        p->pscratch_bytes = persist_scratch_bytes(1);
        p->pscratch.sync = reinterpret_cast<unsigned*>(pscr);
        p->pscratch.queue = reinterpret_cast<int*>(pscr + sizeof(unsigned) * kPersistSyncStride);
        p->pscratch.team_prob = p->pscratch.queue + 1;
        p->pscratch.abort_flag = p->pscratch.queue + 2;
    }
    if (base) {
        s.N = N;
        s.W = W;
        s.variant = p->prm.variant;
        s.cap_f = p->cap_f;
        s.cap_s = p->cap_s;
        s.cap_trees = p->cap_trees;
        s.max_pieces = p->max_pieces;
        s.path_cap = p->path_cap;
        s.eta = p->prm.eta;
        s.res = p->prm.edge_res;
        s.p_new = p->prm.p_new;
        s.p_guided = p->prm.p_guided;
        s.H = p->prm.t_max;
        s.thr_guided = (unsigned)std::ceil(p->prm.p_guided * 16777216.0);
        s.thr_new = (unsigned)std::floor(p->prm.p_new * 16777216.0);
        s.learned = p->prm.learned;
        s.key0 = (unsigned)(p->prm.seed & 0xffffffffull);
        s.key1 = (unsigned)(p->prm.seed >> 32);
        s.problem_id = p->prm.problem_id;
        for (int j = 0; j < kMaxDof; ++j) {
            s.qs[j] = j < p->dof ? (R)p->qs[j] : R(0);
            s.qg[j] = j < p->dof ? (R)p->qg[j] : R(0);
        }
        state_of<R>(p) = s;
    }
    return cv.off;
}

// Plans of this problem run as one persistent launch (STP_LAUNCH_PERSISTENT),
// except with closed-form validation, which only the per-step kernels implement.
bool uses_persistent(const stp_problem* p) {
    return p->prm.launch_mode == STP_LAUNCH_PERSISTENT && !p->prm.continuous;
}

template <typename R>
stp_status create_impl(stp_problem* p) {
    // Sphere order: stable by frame.
    std::vector<int> order(p->S);
    for (int s = 0; s < p->S; ++s) order[s] = s;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return p->sph[5 * a] < p->sph[5 * b]; });
    std::vector<int> link_start(kMaxDof + 2, p->S);
    {
        int nf = p->arm ? p->dof + 1 : 1;
        int s = 0;
        for (int f = 0; f < kMaxDof + 2; ++f) {
            while (s < p->S && (int)p->sph[5 * order[s]] < f) ++s;
            link_start[f] = f < nf ? s : p->S;
            if (f >= nf) link_start[f] = p->S;
        }
        link_start[nf] = p->S;
    }
    compute_self_pairs(p, order);
    int off_way, off_vel, off_rad, off_tim, off_self;
    const size_t blob_bytes = blob_layout<R>(p, &off_way, &off_vel, &off_rad, &off_tim, &off_self);
    R* blob;
    unsigned char* gfree;
    Ctl* ctl;
    R *qdev, *tdev;
    int *cnt, *hit;
    long long* off;
    const size_t bytes = layout_state<R>(p, nullptr, &blob, blob_bytes, &gfree, &ctl, &qdev, &tdev, &cnt, &off, &hit);
    void* arena = nullptr;
    cudaError_t e = cache_alloc(&arena, bytes, &p->arena_block);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaMalloc(arena)");
    p->d_arena = static_cast<char*>(arena);
    p->arena_bytes = bytes;
    layout_state<R>(p, p->d_arena, &blob, blob_bytes, &gfree, &ctl, &qdev, &tdev, &cnt, &off, &hit);
    p->d_ctl = ctl;
    fill_geom<R>(p, geom_of<R>(p), blob, (unsigned)blob_bytes, off_way, off_vel, off_rad, off_tim, off_self,
                 link_start);
    State<R>& S = state_of<R>(p);
    cudaStream_t st = p->stream;
    std::vector<R> hb = blob_host<R>(p, order, blob_bytes, off_way, off_vel, off_rad, off_tim, off_self);
    STP_CUDA(p, cudaMemcpyAsync(blob, hb.data(), blob_bytes, cudaMemcpyHostToDevice, st));
    STP_CUDA(p, cudaMemsetAsync(S.tile_cnt, 0, sizeof(int) * (size_t)(p->prm.n_roots + 1) * kMaxQTiles, st));
    STP_CUDA(p, cudaMemsetAsync(S.btile_cnt, 0, sizeof(int) * 2 * kMaxQTiles, st));

    // Control-block constants computed in double on the host (Eq. goal-time-lower-bound).
    Ctl hc;
    std::memset(&hc, 0, sizeof(hc));
    hc.Lg = p->Lg;
    hc.H = p->prm.t_max;
    hc.dt = p->prm.env_dt;
    hc.kmin = p->kmin;
    hc.kend = p->kend;
    hc.nk = p->nk;
    hc.budget_ns = p->prm.budget_ms > 0 ? (unsigned long long)(p->prm.budget_ms * 1e6) : 0ull;
    hc.done = 1;
    STP_CUDA(p, cudaMemcpyAsync(ctl, &hc, sizeof(Ctl), cudaMemcpyHostToDevice, st));

    // Start check (q_s, 0) and goal checks (q_g, k dt), k = kmin..kmax, in one batch:
    // entry 0 is the start, entries 1..nk the goal grid.
    const int ng = p->nk + 1;
    std::vector<R> hq((size_t)ng * kDP, R(0));
    std::vector<R> ht(ng);
    for (int j = 0; j < p->dof; ++j) hq[j] = (R)p->qs[j];
    ht[0] = R(0);
    for (int i = 0; i < p->nk; ++i) {
        for (int j = 0; j < p->dof; ++j) hq[(size_t)(i + 1) * kDP + j] = (R)p->qg[j];
        ht[i + 1] = (R)((double)(p->kmin + i) * p->prm.env_dt);
    }
    R* qall = nullptr;
    e = cudaMallocAsync(&qall, sizeof(R) * hq.size(), st);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaMallocAsync(goal grid)");
    STP_CUDA(p, cudaMemcpyAsync(qall, hq.data(), sizeof(R) * hq.size(), cudaMemcpyHostToDevice, st));
    STP_CUDA(p, cudaMemcpyAsync(tdev, ht.data(), sizeof(R) * ng, cudaMemcpyHostToDevice, st));
    std::vector<int> hcnt(ng, 1);
    std::vector<long long> hoff(ng + 1);
    for (int i = 0; i <= ng; ++i) hoff[i] = i;
    STP_CUDA(p, cudaMemcpyAsync(cnt, hcnt.data(), sizeof(int) * ng, cudaMemcpyHostToDevice, st));
    STP_CUDA(p, cudaMemcpyAsync(off, hoff.data(), sizeof(long long) * (ng + 1), cudaMemcpyHostToDevice, st));
    STP_CUDA(p, cudaMemsetAsync(hit, 0, sizeof(int) * ng, st));
    EdgeBatch<R> E{};
    E.done = nullptr;
    E.qa = qall;
    E.qb = qall;
    E.ta = tdev;
    E.tb = tdev;
    E.qstride = kDP;
    E.cnt = cnt;
    E.off = off;
    E.n_host = ng;
    E.hit = hit;
    E.err = &ctl->err;
    STP_CUDA(p, launch_validate<R>(geom_of<R>(p), E, false, true, 0, st));
    std::vector<int> hh(ng);
    STP_CUDA(p, cudaMemcpyAsync(hh.data(), hit, sizeof(int) * ng, cudaMemcpyDeviceToHost, st));
    STP_CUDA(p, cudaFreeAsync(qall, st));
    STP_CUDA(p, cudaStreamSynchronize(st));
    p->start_free = hh[0] == 0;
    std::vector<unsigned char> gf(std::max(p->nk, 1), 0);
    for (int i = 0; i < p->nk; ++i) gf[i] = hh[i + 1] == 0 ? 1 : 0;
    // Pageable source: the call returns once the bytes are staged.
    STP_CUDA(p, cudaMemcpyAsync(gfree, gf.data(), gf.size(), cudaMemcpyHostToDevice, st));
    if (uses_persistent(p)) {
        // One team of every resident CTA (or persist_ctas of them).
        p->persist_dq = persist_dq(p->dof);
        p->persist_smem = persist_smem_bytes((int)blob_bytes, p->prm.ext_per_iter);
        int per_sm = 0;
        STP_CUDA(p, persist_blocks_per_sm<R>(p->persist_dq, p->persist_smem, &per_sm, persist_threads(false)));
        if (per_sm < 1) {
            p->last_error = "persistent planner kernel does not fit on an SM";
            g_last_error = p->last_error;
            return STP_ERR_CAPACITY;
        }
        const int resident = validate_grid_blocks() * per_sm;
        p->persist_grid = p->prm.persist_ctas > 0 ? std::min(p->prm.persist_ctas, resident) : resident;
    }
    return STP_OK;
}

template <typename R>
stp_status capture_graph(stp_problem* p) {
    // Default 8: capture and instantiation (or the update of a cached graph)
    // grow with the graph while replays of small graphs cost the device almost
    // nothing (UR5e, 32 iterations, before graphs were cached: one
    // create-plan-free 2.80 ms with 8 against 3.25 ms with 32; plan 2.27 ms
    // against 2.26 ms).
    const int G = p->prm.iters_per_graph > 0 ? p->prm.iters_per_graph : 8;
    const bool prof = p->profiling != 0;
    const bool have_prof = !p->prof_ev.empty();
    if (p->graph && p->graph_stream == p->stream && p->graph_iters == G && prof == have_prof &&
        p->graph_trace == state_of<R>(p).trace)
        return STP_OK;
    if (p->graph) {
        // Graphs holding this problem's profiling events are not kept.
        if (have_prof) cudaGraphExecDestroy(p->graph);
        else cache_graph_release(p->graph);
        p->graph = nullptr;
    }
    for (cudaEvent_t e : p->prof_ev) cudaEventDestroy(e);
    p->prof_ev.clear();
    if (prof) {
        p->prof_ev.resize((size_t)G * (kIterKernels + 1));
        for (auto& e : p->prof_ev) STP_CUDA(p, cudaEventCreate(&e));
    }
    cudaGraph_t g;
    STP_CUDA(p, cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaSuccess;
    for (int i = 0; i < G && err == cudaSuccess; ++i)
        err = launch_iteration<R>(geom_of<R>(p), state_of<R>(p), 0, p->stream,
                                  prof ? &p->prof_ev[(size_t)i * (kIterKernels + 1)] : nullptr);
    cudaError_t e2 = cudaStreamEndCapture(p->stream, &g);
    if (err != cudaSuccess) {
        if (e2 == cudaSuccess) cudaGraphDestroy(g);
        return cuda_fail(p, err, "capture(iteration)");
    }
    if (e2 != cudaSuccess) return cuda_fail(p, e2, "cudaStreamEndCapture");
    err = prof ? cudaGraphInstantiate(&p->graph, g, 0) : cache_graph_exec(g, &p->graph);
    cudaGraphDestroy(g);
    if (err != cudaSuccess) return cuda_fail(p, err, "cudaGraphInstantiate");
    p->graph_iters = G;
    p->graph_stream = p->stream;
    p->graph_trace = state_of<R>(p).trace;
    return STP_OK;
}

template <typename R>
stp_status plan_persistent_impl(stp_problem* p, Ctl* hc) {
    cudaStream_t st = p->stream;
    State<R>& S = state_of<R>(p);
    const int mi = p->prm.max_iters;
    STP_CUDA(p, cudaEventRecord(p->ev_step0, st));
    STP_CUDA(p, cudaMemcpyAsync(p->d_pgeom, &geom_of<R>(p), sizeof(Geom<R>), cudaMemcpyHostToDevice, st));
    STP_CUDA(p, cudaMemcpyAsync(p->d_pstate, &S, sizeof(State<R>), cudaMemcpyHostToDevice, st));
    STP_CUDA(p, cudaMemcpyAsync(p->d_pmax_iters, &mi, sizeof(int), cudaMemcpyHostToDevice, st));
    STP_CUDA(p, cudaMemsetAsync(p->pscratch.sync, 0, p->pscratch_bytes, st));
    if (p->d_trace)
        STP_CUDA(p, cudaMemsetAsync(p->d_trace, 0xff,
                                    sizeof(int) * (size_t)p->trace_iters * p->prm.ext_per_iter * kTraceInts, st));
    STP_CUDA(p, cudaMemsetAsync(S.tile_cnt, 0, sizeof(int) * (size_t)(p->prm.n_roots + 1) * kMaxQTiles, st));
    STP_CUDA(p, cudaMemsetAsync(S.btile_cnt, 0, sizeof(int) * 2 * kMaxQTiles, st));
    PersistArgs<R> a{};
    a.Gs = static_cast<const Geom<R>*>(p->d_pgeom);
    a.Ss = static_cast<const State<R>*>(p->d_pstate);
    a.max_iters = p->d_pmax_iters;
    a.P = 1;
    a.team_size = p->persist_grid;
    a.sync = p->pscratch.sync;
    a.queue = p->pscratch.queue;
    a.team_prob = p->pscratch.team_prob;
    a.abort_flag = p->pscratch.abort_flag;
    STP_CUDA(p, cudaEventRecord(p->ev0, st));
    STP_CUDA(p, launch_plan_persistent<R>(a, p->persist_dq, p->persist_grid, p->persist_smem, st,
                                          persist_threads(false)));
    STP_CUDA(p, cudaEventRecord(p->ev1, st));
    STP_CUDA(p, cudaMemcpyAsync(hc, p->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    STP_CUDA(p, cudaEventRecord(p->ev_step1, st));
    STP_CUDA(p, cudaStreamSynchronize(st));
    // Step times (device global timer, barrier to barrier), in the order of
    // the per-step kernels' profile; the two bridge passes count together.
    static const int kMap[8] = {0, 1, 2, 3, 4, 5, 5, 6};
    for (int k = 0; k < kIterKernels; ++k) {
        p->prof_ms[k] = 0.0;
        p->prof_launches[k] = 0;
    }
    for (int ph = 0; ph < 8; ++ph) p->prof_ms[kMap[ph]] += (double)hc->ph_ns[ph] * 1e-6;
    for (int k = 0; k < kIterKernels; ++k) p->prof_launches[k] = hc->iter;
    return STP_OK;
}

template <typename R>
stp_status plan_impl(stp_problem* p, Ctl* hc) {
    if (uses_persistent(p)) return plan_persistent_impl<R>(p, hc);
    cudaStream_t st = p->stream;
    stp_status s = capture_graph<R>(p);
    if (s != STP_OK) return s;
    const int G = p->graph_iters;
    STP_CUDA(p, cudaEventRecord(p->ev_step0, st));
    if (p->d_trace)
        STP_CUDA(p, cudaMemsetAsync(p->d_trace, 0xff,
                                    sizeof(int) * (size_t)p->trace_iters * p->prm.ext_per_iter * kTraceInts, st));
    STP_CUDA(p, cudaMemsetAsync(state_of<R>(p).tile_cnt, 0,
                                sizeof(int) * (size_t)(p->prm.n_roots + 1) * kMaxQTiles, st));
    STP_CUDA(p, cudaMemsetAsync(state_of<R>(p).btile_cnt, 0, sizeof(int) * 2 * kMaxQTiles, st));
    STP_CUDA(p, cudaEventRecord(p->ev0, st));
    STP_CUDA(p, launch_plan_reset<R>(geom_of<R>(p), state_of<R>(p), p->prm.max_iters, st));
    const int n_launch = (p->prm.max_iters + G - 1) / G;
    auto t0 = std::chrono::steady_clock::now();
    for (int k = 0; k < kIterKernels; ++k) {
        p->prof_ms[k] = 0.0;
        p->prof_launches[k] = 0;
    }
    int iters_before = 0;
    for (int i = 0; i < n_launch; ++i) {
        STP_CUDA(p, cudaGraphLaunch(p->graph, st));
        if (p->profiling) {
            int iters_after = 0;
            STP_CUDA(p, cudaMemcpyAsync(&iters_after, &p->d_ctl->iter, sizeof(int), cudaMemcpyDeviceToHost, st));
            STP_CUDA(p, cudaStreamSynchronize(st));
            const int ran = std::min(p->graph_iters, iters_after - iters_before);
            for (int it = 0; it < ran; ++it) {
                cudaEvent_t* ev = &p->prof_ev[(size_t)it * (kIterKernels + 1)];
                for (int k = 0; k < kIterKernels; ++k) {
                    float ms = 0.f;
                    STP_CUDA(p, cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
                    p->prof_ms[k] += ms;
                    p->prof_launches[k] += 1;
                }
            }
            iters_before = iters_after;
        }
        if (p->prm.budget_ms > 0) {
            STP_CUDA(p, cudaStreamSynchronize(st));
            double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            if (ms >= p->prm.budget_ms) break;
        }
    }
    STP_CUDA(p, cudaEventRecord(p->ev1, st));
    STP_CUDA(p, launch_extract_path<R>(state_of<R>(p), p->dof, st));
    STP_CUDA(p, cudaMemcpyAsync(hc, p->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    STP_CUDA(p, cudaEventRecord(p->ev_step1, st));
    STP_CUDA(p, cudaStreamSynchronize(st));
    return STP_OK;
}

template <typename R>
stp_status copy_path(stp_problem* p, int n, double* path, int cap) {
    if (n > cap) return STP_ERR_CAPACITY;
    std::vector<R> h((size_t)n * kDP);
    STP_CUDA(p, cudaMemcpy(h.data(), state_of<R>(p).path, sizeof(R) * h.size(), cudaMemcpyDeviceToHost));
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < p->dof; ++j) path[(size_t)i * (p->dof + 1) + j] = (double)h[(size_t)i * kDP + j];
        path[(size_t)i * (p->dof + 1) + p->dof] = (double)h[(size_t)i * kDP + kDP - 1];
    }
    return STP_OK;
}

template <typename R>
stp_status check_edges_impl(stp_problem* p, int n, const void* qa, const void* ta, const void* qb, const void* tb,
                            int flags, unsigned char* verdict, void* min_clearance, int* n_checks) {
    cudaStream_t st = p->stream;
    const bool dev = (flags & STP_EDGES_DEVICE) != 0;
    const bool clear = (flags & STP_EDGES_CLEARANCE) != 0;
    const bool early = (flags & STP_EDGES_NO_EARLY_EXIT) == 0;
    const int d = p->dof;
    Carver cv;
    auto lay = [&](char* base) {
        cv.off = 0;
        cv.base = base;
        struct L {
            R *qa, *qb, *ta, *tb, *clr;
            int *cnt, *hit;
            long long *off, *tmp;
            unsigned char* ver;
        } l;
        l.qa = dev ? nullptr : cv.take<R>((size_t)n * d);
        l.qb = dev ? nullptr : cv.take<R>((size_t)n * d);
        l.ta = dev ? nullptr : cv.take<R>(n);
        l.tb = dev ? nullptr : cv.take<R>(n);
        l.cnt = cv.take<int>(n);
        l.off = cv.take<long long>((size_t)n + 1);
        l.tmp = cv.take<long long>((size_t)n / 4096 + 2);
        l.hit = cv.take<int>((size_t)n + 1);  // flags, then the window counter
        l.clr = clear ? cv.take<R>(n) : nullptr;
        l.ver = dev ? nullptr : cv.take<unsigned char>(n);
        return l;
    };
    lay(nullptr);
    if (cv.off > p->scratch_bytes) {
        // The previous scratch is idle: every check ends with a stream synchronisation.
        cache_release(p->d_scratch, p->scratch_bytes);
        p->d_scratch = nullptr;
        p->scratch_bytes = 0;
        void* sc = nullptr;
        size_t got = 0;
        cudaError_t e = cache_alloc(&sc, cv.off, &got);
        if (e != cudaSuccess) return cuda_fail(p, e, "cudaMalloc(edge scratch)");
        p->d_scratch = static_cast<char*>(sc);
        p->scratch_bytes = got;
    }
    auto L = lay(p->d_scratch);
    const R* dqa = dev ? (const R*)qa : L.qa;
    const R* dqb = dev ? (const R*)qb : L.qb;
    const R* dta = dev ? (const R*)ta : L.ta;
    const R* dtb = dev ? (const R*)tb : L.tb;
    if (!dev) {
        STP_CUDA(p, cudaMemcpyAsync(L.qa, qa, sizeof(R) * n * d, cudaMemcpyHostToDevice, st));
        STP_CUDA(p, cudaMemcpyAsync(L.qb, qb, sizeof(R) * n * d, cudaMemcpyHostToDevice, st));
        STP_CUDA(p, cudaMemcpyAsync(L.ta, ta, sizeof(R) * n, cudaMemcpyHostToDevice, st));
        STP_CUDA(p, cudaMemcpyAsync(L.tb, tb, sizeof(R) * n, cudaMemcpyHostToDevice, st));
    }
    STP_CUDA(p, launch_edge_counts<R>(geom_of<R>(p), dqa, dta, dqb, dtb, d, n, p->prm.edge_res, L.cnt, st));
    STP_CUDA(p, launch_scan_counts(L.cnt, n, L.off, L.tmp, st));
    STP_CUDA(p, cudaMemsetAsync(L.hit, 0, sizeof(int) * ((size_t)n + 1), st));
    if (clear) {
        unsigned long long inf_bits = sizeof(R) == 4 ? 0x7f800000ull : 0x7ff0000000000000ull;
        STP_CUDA(p, launch_fill(L.clr, n, (int)sizeof(R), inf_bits, st));
    }
    EdgeBatch<R> E{};
    E.qa = dqa;
    E.qb = dqb;
    E.ta = dta;
    E.tb = dtb;
    E.qstride = d;
    E.cnt = L.cnt;
    E.off = L.off;
    E.n_host = n;
    E.hit = L.hit;
    E.win_next = L.hit + n;
    E.clear = L.clr;
    E.err = &p->d_ctl->err;
    STP_CUDA(p, cudaMemsetAsync(p->d_counters, 0, 2 * sizeof(unsigned long long), st));
    E.points_done = p->d_counters;
    E.pairs_done = p->d_counters + 1;
    STP_CUDA(p, cudaEventRecord(p->ev2, st));
    STP_CUDA(p, launch_validate<R>(geom_of<R>(p), E, clear, early, 0, st));
    STP_CUDA(p, cudaEventRecord(p->ev3, st));
    unsigned char* dver = dev ? verdict : L.ver;
    R* dclr = clear ? (dev ? (R*)min_clearance : L.clr) : nullptr;
    if (clear && dev) {
        STP_CUDA(p, cudaMemcpyAsync(dclr, L.clr, sizeof(R) * n, cudaMemcpyDeviceToDevice, st));
    }
    STP_CUDA(p, launch_finish_batch<R>(n, L.hit, dver, dclr, st));
    if (!dev) {
        STP_CUDA(p, cudaMemcpyAsync(verdict, L.ver, n, cudaMemcpyDeviceToHost, st));
        if (clear && min_clearance)
            STP_CUDA(p, cudaMemcpyAsync(min_clearance, L.clr, sizeof(R) * n, cudaMemcpyDeviceToHost, st));
        if (n_checks) STP_CUDA(p, cudaMemcpyAsync(n_checks, L.cnt, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
        STP_CUDA(p, cudaStreamSynchronize(st));
    } else if (n_checks) {
        STP_CUDA(p, cudaMemcpyAsync(n_checks, L.cnt, sizeof(int) * n, cudaMemcpyDeviceToDevice, st));
    }
    return STP_OK;
}

}  // namespace

extern "C" {

const char* stp_status_string(stp_status s) {
    switch (s) {
        case STP_OK: return "STP_OK";
        case STP_ERR_INVALID: return "STP_ERR_INVALID";
        case STP_ERR_CAPACITY: return "STP_ERR_CAPACITY";
        case STP_ERR_CUDA: return "STP_ERR_CUDA";
        case STP_ERR_TIMEOUT: return "STP_ERR_TIMEOUT";
        case STP_NO_SOLUTION: return "STP_NO_SOLUTION";
    }
    return "STP_UNKNOWN";
}

const char* stp_last_error(const stp_problem* p) { return p ? p->last_error.c_str() : g_last_error.c_str(); }

stp_status stp_create_problem(const stp_robot* robot, const stp_obstacles* obs, const double* q_start,
                              const double* q_goal, const stp_params* params, stp_problem** out) {
    clear_stale_error();
    if (!out) return STP_ERR_INVALID;
    *out = nullptr;
    if (!robot || !obs || !q_start || !q_goal || !params) return STP_ERR_INVALID;
    const int d = robot->dof;
    if (d < 2 || d > kMaxDof) return STP_ERR_INVALID;
    if (!robot->arm && d > 3) return STP_ERR_INVALID;
    if (robot->arm && !robot->dh) return STP_ERR_INVALID;
    if (!robot->q_lo || !robot->q_hi || !robot->spheres) return STP_ERR_INVALID;
    if (robot->n_spheres < 1 || robot->n_spheres > kMaxSpheres) return STP_ERR_INVALID;
    if (!(robot->v_max > 0) || !std::isfinite(robot->v_max)) return STP_ERR_INVALID;
    if (obs->n_obs < 0 || obs->n_obs > kMaxObs || obs->n_way < 1 || obs->n_way > kMaxWay) return STP_ERR_INVALID;
    if (obs->n_obs > 0 && (!obs->radius || !obs->way)) return STP_ERR_INVALID;
    const stp_params& P = *params;
    if (P.variant < 0 || P.variant > 2) return STP_ERR_INVALID;
    if (P.n_roots < 1 || P.n_roots > kMaxRoots) return STP_ERR_INVALID;
    if (P.ext_per_iter < 1 || P.ext_per_iter > kMaxWorkers) return STP_ERR_INVALID;
    if (P.max_iters < 1) return STP_ERR_INVALID;
    if (!(P.eta > 0) || !(P.edge_res > 0) || !(P.env_dt > 0) || !(P.t_max > 0)) return STP_ERR_INVALID;
    if (!(P.p_new >= 0 && P.p_new <= 1) || !(P.p_guided >= 0 && P.p_guided <= 1)) return STP_ERR_INVALID;
    if (P.precision != 0 && P.precision != 1) return STP_ERR_INVALID;
    if ((P.learned != 0 && P.learned != 1) || P.capacity < 0 || P.iters_per_graph < 0) return STP_ERR_INVALID;
    if (P.launch_mode < STP_LAUNCH_DEFAULT || P.launch_mode > STP_LAUNCH_PERSISTENT || P.persist_ctas < 0)
        return STP_ERR_INVALID;
    if (!(P.t_offset >= 0) || !std::isfinite(P.t_offset)) return STP_ERR_INVALID;
    if (P.continuous != 0 && (P.continuous != 1 || robot->arm)) return STP_ERR_INVALID;
    if (P.self_collision != 0 && (P.self_collision != 1 || !robot->arm)) return STP_ERR_INVALID;

    stp_problem* p = new (std::nothrow) stp_problem();
    if (!p) return STP_ERR_CUDA;
    p->precision = P.precision;
    p->prm = P;
    p->dof = d;
    p->arm = robot->arm ? 1 : 0;
    p->S = robot->n_spheres;
    p->M = obs->n_obs;
    p->K = obs->n_way;
    p->vmax = robot->v_max;
    p->qs.assign(q_start, q_start + d);
    p->qg.assign(q_goal, q_goal + d);
    p->qlo.assign(robot->q_lo, robot->q_lo + d);
    p->qhi.assign(robot->q_hi, robot->q_hi + d);
    if (p->arm) p->dh.assign(robot->dh, robot->dh + 4 * d);
    p->sph.assign(robot->spheres, robot->spheres + 5 * p->S);
    if (p->M > 0) {
        p->obs_r.assign(obs->radius, obs->radius + p->M);
        p->way.assign(obs->way, obs->way + (size_t)p->M * p->K * 4);
        // Local query time 0 is absolute time t_offset: shift the trajectories.
        for (size_t i = 0; i < p->way.size(); i += 4) p->way[i] -= P.t_offset;
    }
    bool ok = finite_all(p->qs.data(), d) && finite_all(p->qg.data(), d) && finite_all(p->qlo.data(), d) &&
              finite_all(p->qhi.data(), d) && finite_all(p->sph.data(), p->sph.size()) &&
              finite_all(p->obs_r.data(), p->obs_r.size()) && finite_all(p->way.data(), p->way.size()) &&
              finite_all(p->dh.data(), p->dh.size());
    for (int j = 0; j < d && ok; ++j) ok = p->qlo[j] <= p->qhi[j];
    for (int s = 0; s < p->S && ok; ++s) {
        double f = p->sph[5 * s];
        ok = f == std::floor(f) && f >= 0 && f <= (p->arm ? d : 0) && p->sph[5 * s + 4] >= 0;
    }
    for (int m = 0; m < p->M && ok; ++m) {
        ok = p->obs_r[m] >= 0;
        for (int k = 1; k < p->K && ok; ++k)
            ok = p->way[((size_t)m * p->K + k) * 4] > p->way[((size_t)m * p->K + k - 1) * 4];
    }
    if (!ok) {
        delete p;
        return STP_ERR_INVALID;
    }
    // Eq. goal-time-lower-bound.
    p->Lg = host_dist(p->qs.data(), p->qg.data(), d) / p->vmax;
    p->kmin = (long long)std::ceil(p->Lg / P.env_dt);
    p->kmax = (long long)std::floor(P.t_max / P.env_dt);
    long long nk = p->kmax - p->kmin + 1;
    if (nk < 0) nk = 0;
    if (nk > (1LL << 24)) {
        delete p;
        return STP_ERR_CAPACITY;
    }
    p->nk = (int)nk;
    p->kend = p->kmin;
    while ((double)p->kend * P.env_dt < P.t_max) ++p->kend;
    const long long half = (P.ext_per_iter + 1) / 2;
    long long cap = P.capacity > 0 ? P.capacity : (long long)P.max_iters * half + 2;
    long long cap_s = P.capacity > 0 ? P.capacity : 2 * (long long)P.max_iters * half + 2;
    if (cap > (1LL << 30) || cap_s * P.n_roots > (1LL << 31)) {
        delete p;
        return STP_ERR_CAPACITY;
    }
    p->cap_f = (int)cap;
    p->cap_s = (int)cap_s;
    p->cap_trees = P.variant == 0 ? (int)std::min<long long>(cap_s * P.n_roots / 2 + 1, 1 << 26) : 1;
    p->max_pieces = std::max(p->nk, 1) + P.n_roots + 1;
    p->path_cap = (int)std::min<long long>(cap + cap_s, 1 << 20);

    int dev_count = 0;
    cudaError_t e = cudaGetDeviceCount(&dev_count);
    if (e != cudaSuccess || dev_count == 0) {
        g_last_error = "no CUDA device";
        delete p;
        return STP_ERR_CUDA;
    }
    e = cache_stream(&p->own_stream);
    if (e != cudaSuccess) {
        cuda_fail(p, e, "cudaStreamCreateWithFlags");
        delete p;
        return STP_ERR_CUDA;
    }
    p->stream = p->own_stream;
    cudaEventCreate(&p->ev0);
    cudaEventCreate(&p->ev1);
    cudaEventCreate(&p->ev2);
    cudaEventCreate(&p->ev3);
    cudaEventCreate(&p->ev_step0);
    cudaEventCreate(&p->ev_step1);
    void* counters = nullptr;
    e = cache_alloc(&counters, 2 * sizeof(unsigned long long), &p->counters_block);
    p->d_counters = static_cast<unsigned long long*>(counters);
    if (e != cudaSuccess) {
        cuda_fail(p, e, "cudaMalloc(counters)");
        stp_free(p);
        return STP_ERR_CUDA;
    }
    stp_status s = p->precision == 0 ? create_impl<float>(p) : create_impl<double>(p);
    if (s != STP_OK) {
        stp_free(p);
        return s;
    }
    *out = p;
    return STP_OK;
}

stp_status stp_set_stream(stp_problem* p, void* cuda_stream) {
    if (!p) return STP_ERR_INVALID;
    p->stream = cuda_stream ? (cudaStream_t)cuda_stream : p->own_stream;
    return STP_OK;
}

stp_status stp_plan(stp_problem* p, double* arrival_U, double* length_C, int* n_path, double* path, int cap,
                    stp_stats* stats) {
    clear_stale_error();
    if (!p) return STP_ERR_INVALID;
    if (path && cap < 0) return STP_ERR_INVALID;
    stp_stats st;
    std::memset(&st, 0, sizeof(st));
    st.first_solution_iter = -1;
    st.U = kInfD;
    st.C = kInfD;
    if (p->prm.learned && !p->has_proposal) {
        p->last_error = "learned sampling needs a proposal (stp_set_proposal)";
        g_last_error = p->last_error;
        return STP_ERR_INVALID;
    }
    const int d = p->dof;
    bool same = true;
    for (int j = 0; j < d; ++j) same = same && p->qs[j] == p->qg[j];
    stp_status result;
    int np = 0;
    if (!p->start_free) {
        result = STP_NO_SOLUTION;
    } else if (same) {
        // First line of Algorithms 2 and 3: q_s = q_g and x_s free.
        st.U = 0.0;
        st.C = 0.0;
        st.first_solution_iter = 0;
        np = 1;
        if (path) {
            if (cap < 1) return STP_ERR_CAPACITY;
            for (int j = 0; j < d; ++j) path[j] = p->qs[j];
            path[d] = 0.0;
        }
        result = STP_OK;
    } else {
        Ctl hc;
        stp_status s = p->precision == 0 ? plan_impl<float>(p, &hc) : plan_impl<double>(p, &hc);
        if (s != STP_OK) return s;
        p->planned = true;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p->ev0, p->ev1);
        st.plan_ms = ms;
        float sms = 0.f;
        cudaEventElapsedTime(&sms, p->ev_step0, p->ev_step1);
        st.step_ms = sms;
        st.iterations = hc.iter;
        st.first_solution_iter = hc.first_iter;
        st.nodes = (long long)hc.st_ins;
        st.edges_validated = (long long)hc.st_ext;
        st.bridges_validated = (long long)hc.st_bridge;
        st.root_checks = (long long)hc.st_root;
        st.check_points = (long long)hc.st_points;
        st.pair_tests = (long long)hc.st_pairs;
        st.nn_evals = (long long)hc.st_nn_evals;
        st.nn_nodes = (long long)hc.st_nn_nodes;
        st.bridge_evals = (long long)hc.st_br_evals;
        st.bridge_nodes = (long long)hc.st_br_nodes;
        st.first_solution_ms = hc.first_iter >= 0 ? (double)(hc.t_first - hc.t_start) * 1e-6 : -1.0;
        st.U = hc.U;
        st.C = hc.C;
        if (hc.err & kErrCapacity) return STP_ERR_CAPACITY;
        if (hc.err & kErrTimeout) return STP_ERR_TIMEOUT;
        if (hc.err) return STP_ERR_CUDA;
        int len = 0;
        STP_CUDA(p, cudaMemcpy(&len, p->precision == 0 ? p->sf.path_len : p->sd.path_len, sizeof(int),
                               cudaMemcpyDeviceToHost));
        if (len < 0) return STP_ERR_CAPACITY;
        np = len;
        if (path && np > 0) {
            stp_status cs = p->precision == 0 ? copy_path<float>(p, np, path, cap) : copy_path<double>(p, np, path, cap);
            if (cs != STP_OK) return cs;
        }
        result = hc.first_iter >= 0 ? STP_OK : STP_NO_SOLUTION;
    }
    if (arrival_U) *arrival_U = st.U;
    if (length_C) *length_C = st.C;
    if (n_path) *n_path = np;
    if (stats) *stats = st;
    return result;
}

stp_status stp_check_edges(stp_problem* p, int n_edges, const void* qa, const void* ta, const void* qb,
                           const void* tb, int flags, unsigned char* verdict, void* min_clearance, int* n_checks) {
    clear_stale_error();
    if (!p || n_edges < 0 || n_edges > (1 << 26)) return STP_ERR_INVALID;
    if (n_edges == 0) return STP_OK;
    if (!qa || !ta || !qb || !tb || !verdict) return STP_ERR_INVALID;
    if (min_clearance && !(flags & STP_EDGES_CLEARANCE)) return STP_ERR_INVALID;
    return p->precision == 0
               ? check_edges_impl<float>(p, n_edges, qa, ta, qb, tb, flags, verdict, min_clearance, n_checks)
               : check_edges_impl<double>(p, n_edges, qa, ta, qb, tb, flags, verdict, min_clearance, n_checks);
}

void stp_release_cached(void) {
    DevCache& c = dev_cache();
    std::lock_guard<std::mutex> g(c.mu);
    int prev = 0;
    cudaGetDevice(&prev);
    for (auto& kv : c.blocks) {
        cudaSetDevice(kv.second.dev);
        cudaFree(kv.second.ptr);
    }
    c.blocks.clear();
    c.cached = 0;
    for (auto& ds : c.streams) {
        cudaSetDevice(ds.first);
        cudaStreamDestroy(ds.second);
    }
    c.streams.clear();
    for (auto& dg : c.graphs) {
        cudaSetDevice(dg.first);
        cudaGraphExecDestroy(dg.second);
    }
    c.graphs.clear();
    cudaSetDevice(prev);
}

void stp_free(stp_problem* p) {
    if (!p) return;
    // Every buffer goes back to the cache idle: wait for the problem's streams.
    if (p->stream) cudaStreamSynchronize(p->stream);
    if (p->own_stream && p->own_stream != p->stream) cudaStreamSynchronize(p->own_stream);
    if (p->graph) {
        if (p->prof_ev.empty()) cache_graph_release(p->graph);
        else cudaGraphExecDestroy(p->graph);
    }
    cache_release(p->d_arena, p->arena_block);
    cache_release(p->d_scratch, p->scratch_bytes);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    if (p->ev2) cudaEventDestroy(p->ev2);
    if (p->ev3) cudaEventDestroy(p->ev3);
    if (p->ev_step0) cudaEventDestroy(p->ev_step0);
    if (p->ev_step1) cudaEventDestroy(p->ev_step1);
    cache_stream_release(p->own_stream);
    cache_release(p->d_counters, p->counters_block);
    for (cudaEvent_t e : p->prof_ev) cudaEventDestroy(e);
    if (p->d_trace) cudaFree(p->d_trace);
    delete p;
}

stp_status stp_set_trace(stp_problem* p, int max_iters) {
    clear_stale_error();
    if (!p || max_iters < 0) return STP_ERR_INVALID;
    if (p->stream) STP_CUDA(p, cudaStreamSynchronize(p->stream));
    if (p->d_trace) {
        STP_CUDA(p, cudaFree(p->d_trace));
        p->d_trace = nullptr;
    }
    p->trace_iters = std::min(max_iters, std::max(p->prm.max_iters, 1));
    if (p->trace_iters > 0) {
        const size_t bytes = sizeof(int) * (size_t)p->trace_iters * p->prm.ext_per_iter * kTraceInts;
        STP_CUDA(p, cudaMalloc(&p->d_trace, bytes));
        STP_CUDA(p, cudaMemset(p->d_trace, 0xff, bytes));
    }
    p->sf.trace = p->sd.trace = p->d_trace;
    p->sf.trace_iters = p->sd.trace_iters = p->d_trace ? p->trace_iters : 0;
    return STP_OK;
}

stp_status stp_trace(stp_problem* p, int* records, int cap_iters, int* n_iters) {
    clear_stale_error();
    if (!p || !n_iters || cap_iters < 0) return STP_ERR_INVALID;
    *n_iters = 0;
    if (!p->d_trace || !p->planned) return STP_OK;
    Ctl hc;
    STP_CUDA(p, cudaStreamSynchronize(p->stream));
    STP_CUDA(p, cudaMemcpy(&hc, p->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    const int n = std::min(hc.iter, p->trace_iters);
    *n_iters = n;
    if (!records) return STP_OK;
    if (cap_iters < n) return STP_ERR_CAPACITY;
    STP_CUDA(p, cudaMemcpy(records, p->d_trace, sizeof(int) * (size_t)n * p->prm.ext_per_iter * kTraceInts,
                           cudaMemcpyDeviceToHost));
    return STP_OK;
}

stp_status stp_last_validate(stp_problem* p, double* ms, long long* points, long long* pairs) {
    if (!p) return STP_ERR_INVALID;
    STP_CUDA(p, cudaStreamSynchronize(p->stream));
    if (ms) {
        float f = 0.f;
        STP_CUDA(p, cudaEventElapsedTime(&f, p->ev2, p->ev3));
        *ms = f;
    }
    unsigned long long c[2];
    STP_CUDA(p, cudaMemcpy(c, p->d_counters, sizeof(c), cudaMemcpyDeviceToHost));
    if (points) *points = (long long)c[0];
    if (pairs) *pairs = (long long)c[1];
    return STP_OK;
}

stp_status stp_set_profiling(stp_problem* p, int on) {
    if (!p) return STP_ERR_INVALID;
    p->profiling = on ? 1 : 0;
    return STP_OK;
}

stp_status stp_profile(stp_problem* p, int cap, const char** names, double* ms, long long* launches, int* n) {
    if (!p || !n) return STP_ERR_INVALID;
    *n = std::min(cap, kIterKernels);
    for (int k = 0; k < *n; ++k) {
        if (names) names[k] = kIterKernelNames[k];
        if (ms) ms[k] = p->prof_ms[k];
        if (launches) launches[k] = p->prof_launches[k];
    }
    return STP_OK;
}

stp_status stp_tree_size(stp_problem* p, int arena, int* n) {
    if (!p || !n || arena < -1 || arena >= p->prm.n_roots) return STP_ERR_INVALID;
    if (!p->planned) {
        *n = 0;
        return STP_OK;
    }
    Ctl hc;
    STP_CUDA(p, cudaMemcpy(&hc, p->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    *n = arena < 0 ? hc.n_f : hc.n_s[arena];
    return STP_OK;
}

}  // extern "C"

namespace {
template <typename R>
stp_status tree_nodes_impl(stp_problem* p, int arena, int n, double* x, int* parent, double* troot, double* cost,
                           int* tree, int* iter) {
    State<R>& S = state_of<R>(p);
    const size_t o = arena < 0 ? 0 : (size_t)arena * S.cap_s;
    std::vector<R> hx((size_t)n * kDP), hc(n), ht(n);
    std::vector<int> hp(n), htr(n), hi(n);
    const R* bx = arena < 0 ? S.fx : S.bx + o * kDP;
    STP_CUDA(p, cudaMemcpy(hx.data(), bx, sizeof(R) * hx.size(), cudaMemcpyDeviceToHost));
    STP_CUDA(p, cudaMemcpy(hp.data(), arena < 0 ? S.fpar : S.bpar + o, sizeof(int) * n, cudaMemcpyDeviceToHost));
    STP_CUDA(p, cudaMemcpy(hc.data(), arena < 0 ? S.fcost : S.bcost + o, sizeof(R) * n, cudaMemcpyDeviceToHost));
    STP_CUDA(p, cudaMemcpy(hi.data(), arena < 0 ? S.fiter : S.biter + o, sizeof(int) * n, cudaMemcpyDeviceToHost));
    if (arena >= 0) {
        STP_CUDA(p, cudaMemcpy(ht.data(), S.btroot + o, sizeof(R) * n, cudaMemcpyDeviceToHost));
        STP_CUDA(p, cudaMemcpy(htr.data(), S.btree + o, sizeof(int) * n, cudaMemcpyDeviceToHost));
    }
    const int d = p->dof;
    for (int i = 0; i < n; ++i) {
        if (x) {
            for (int j = 0; j < d; ++j) x[(size_t)i * (d + 1) + j] = (double)hx[(size_t)i * kDP + j];
            x[(size_t)i * (d + 1) + d] = (double)hx[(size_t)i * kDP + kDP - 1];
        }
        if (parent) parent[i] = hp[i];
        if (cost) cost[i] = (double)hc[i];
        if (iter) iter[i] = hi[i];
        if (troot) troot[i] = arena < 0 ? 0.0 : (double)ht[i];
        if (tree) tree[i] = arena < 0 ? 0 : htr[i];
    }
    return STP_OK;
}
}  // namespace

extern "C" {

stp_status stp_tree_nodes(stp_problem* p, int arena, double* x, int* parent, double* troot, double* cost, int* tree,
                          int* iter) {
    int n = 0;
    stp_status s = stp_tree_size(p, arena, &n);
    if (s != STP_OK || n == 0) return s;
    return p->precision == 0 ? tree_nodes_impl<float>(p, arena, n, x, parent, troot, cost, tree, iter)
                             : tree_nodes_impl<double>(p, arena, n, x, parent, troot, cost, tree, iter);
}

stp_status stp_history(stp_problem* p, double* U_hist, int cap, int* n) {
    if (!p || !n) return STP_ERR_INVALID;
    *n = 0;
    if (!p->planned) return STP_OK;
    Ctl hc;
    STP_CUDA(p, cudaMemcpy(&hc, p->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    *n = hc.iter;
    if (U_hist && cap > 0) {
        const double* src = p->precision == 0 ? p->sf.U_hist : p->sd.U_hist;
        STP_CUDA(p, cudaMemcpy(U_hist, src, sizeof(double) * std::min(cap, hc.iter), cudaMemcpyDeviceToHost));
    }
    return STP_OK;
}

stp_status stp_slots(stp_problem* p, double* T, int* has_root, int* active, int* gen) {
    if (!p) return STP_ERR_INVALID;
    Ctl hc;
    STP_CUDA(p, cudaMemcpy(&hc, p->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    for (int i = 0; i < p->prm.n_roots; ++i) {
        if (T) T[i] = hc.slot_T[i];
        if (has_root) has_root[i] = hc.slot_has[i];
        if (active) active[i] = hc.slot_active[i];
        if (gen) gen[i] = hc.slot_gen[i];
    }
    return STP_OK;
}

stp_status stp_goal_grid(stp_problem* p, long* kmin, int* n, unsigned char* free_flags, int cap) {
    if (!p || !kmin || !n) return STP_ERR_INVALID;
    *kmin = (long)p->kmin;
    *n = p->nk;
    if (free_flags && cap > 0 && p->nk > 0) {
        const unsigned char* src = p->precision == 0 ? p->sf.gfree : p->sd.gfree;
        STP_CUDA(p, cudaMemcpy(free_flags, src, std::min(cap, p->nk), cudaMemcpyDeviceToHost));
    }
    return STP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Collision batch without allocation (stp_check_edges_noalloc).
// ---------------------------------------------------------------------------
namespace {

constexpr size_t ce_align(size_t x) { return (x + 255) / 256 * 256; }
constexpr int kNoAllocMaxEdges = STP_NOALLOC_MAX_EDGES;
constexpr size_t kNoAllocCnt = 0;
constexpr size_t kNoAllocOff = kNoAllocCnt + ce_align(sizeof(int) * kNoAllocMaxEdges);
constexpr size_t kNoAllocHit = kNoAllocOff + ce_align(sizeof(long long) * (kNoAllocMaxEdges + 1));
constexpr size_t kNoAllocTmp = kNoAllocHit + ce_align(sizeof(int) * (kNoAllocMaxEdges + 1));
constexpr size_t kNoAllocBytes = kNoAllocTmp + ce_align(sizeof(long long) * (kNoAllocMaxEdges / 4096 + 2));
constexpr int kNoAllocMaxDevices = 64;

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

}  // namespace

// Scratch of the allocation-free batch: check counts, offsets, hit flags and
// scan partials for up to STP_NOALLOC_MAX_EDGES edges. In host code this name
// is only a handle; its device address is looked up per device below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

// Device address of the static scratch on the current device (looked up once
// per device, with that device current).
stp_status noalloc_scratch(stp_problem* p, char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices) return STP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return cuda_fail(p, e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_ptr[dev] = ptr;
    }
    *out = static_cast<char*>(g_noalloc_ptr[dev]);
    return STP_OK;
}

template <typename R>
stp_status check_edges_noalloc_impl(stp_problem* p, int n, const void* qa, const void* ta, const void* qb,
                                    const void* tb, unsigned char* verdict) {
    char* base = nullptr;
    stp_status s = noalloc_scratch(p, &base);
    if (s != STP_OK) return s;
    cudaStream_t st = p->stream;
    int* cnt = reinterpret_cast<int*>(base + kNoAllocCnt);
    long long* off = reinterpret_cast<long long*>(base + kNoAllocOff);
    int* hit = reinterpret_cast<int*>(base + kNoAllocHit);
    long long* tmp = reinterpret_cast<long long*>(base + kNoAllocTmp);
    const R* dqa = static_cast<const R*>(qa);
    const R* dqb = static_cast<const R*>(qb);
    const R* dta = static_cast<const R*>(ta);
    const R* dtb = static_cast<const R*>(tb);
    STP_CUDA(p, launch_edge_counts<R>(geom_of<R>(p), dqa, dta, dqb, dtb, p->dof, n, p->prm.edge_res, cnt, st));
    STP_CUDA(p, launch_scan_counts(cnt, n, off, tmp, st));
    // The array keeps the previous call's flags (and window counter after
    // them): clear them.
    STP_CUDA(p, cudaMemsetAsync(hit, 0, sizeof(int) * ((size_t)n + 1), st));
    EdgeBatch<R> E{};
    E.qa = dqa;
    E.qb = dqb;
    E.ta = dta;
    E.tb = dtb;
    E.qstride = p->dof;
    E.cnt = cnt;
    E.off = off;
    E.n_host = n;
    E.hit = hit;
    E.win_next = hit + n;
    E.err = &p->d_ctl->err;
    STP_CUDA(p, launch_validate<R>(geom_of<R>(p), E, false, true, 0, st));
    STP_CUDA(p, launch_finish_batch<R>(n, hit, verdict, nullptr, st));
    return STP_OK;
}

}  // namespace

extern "C" stp_status stp_check_edges_noalloc(stp_problem* p, int n_edges, const void* qa, const void* ta,
                                              const void* qb, const void* tb, unsigned char* verdict) {
    clear_stale_error();
    if (!p || n_edges < 0) return STP_ERR_INVALID;
    if (n_edges > kNoAllocMaxEdges) return STP_ERR_CAPACITY;
    if (n_edges == 0) return STP_OK;
    if (!qa || !ta || !qb || !tb || !verdict) return STP_ERR_INVALID;
    return p->precision == 0 ? check_edges_noalloc_impl<float>(p, n_edges, qa, ta, qb, tb, verdict)
                             : check_edges_noalloc_impl<double>(p, n_edges, qa, ta, qb, tb, verdict);
}

// ---------------------------------------------------------------------------
// Batched planning.
// ---------------------------------------------------------------------------
struct stp_batch {
    int launch_mode = 0;          // 0 persistent work queue, 1 one kernel per step
    int team_ctas = 8;
    int persist_grid = 0, persist_smem = 0;
    PersistScratch scratch{};
    void* d_scratch = nullptr;
    size_t scratch_bytes = 0;
    bool graph_direct = false;    // the cooperative launch could not be captured: launch it directly
    std::vector<stp_problem*> probs;
    std::vector<int*> traces;  // each member's trace buffer when the batch was created
    std::vector<int> trivial;  // 0 plan, 1 blocked start, 2 start == goal
    Geom<float>* d_geom = nullptr;
    State<float>* d_state = nullptr;
    int* d_iters = nullptr;
    BatchShape shape{};
    int iters_per_graph = 16;
    int max_iters = 0;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<Ctl> ctl;
    std::string last_error;
};

// ---------------------------------------------------------------------------
// Learned proposal: network output -> sampler table; problem summary.
// ---------------------------------------------------------------------------
template <typename R>
static stp_status set_proposal_impl(stp_problem* p, const float* y, int flags) {
    State<R>& S = state_of<R>(p);
    STP_CUDA(p, cudaMemcpyAsync(S.prop_y, y, sizeof(float) * kPropY,
                                (flags & STP_MLP_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                p->stream));
    STP_CUDA(p, launch_set_proposal<R>(geom_of<R>(p), S, p->stream));
    STP_CUDA(p, cudaStreamSynchronize(p->stream));
    return STP_OK;
}

extern "C" stp_status stp_set_proposal(stp_problem* p, const float* y, int flags) {
    clear_stale_error();
    if (!p || !y || (flags & ~STP_MLP_DEVICE)) return STP_ERR_INVALID;
    if (!(flags & STP_MLP_DEVICE)) {
        for (int i = 0; i < kPropY; ++i)
            if (!std::isfinite(y[i])) return STP_ERR_INVALID;
    }
    stp_status s = p->precision == 0 ? set_proposal_impl<float>(p, y, flags) : set_proposal_impl<double>(p, y, flags);
    if (s == STP_OK) p->has_proposal = true;
    return s;
}

template <typename R>
static stp_status targets_impl(stp_problem* p, float* t) {
    State<R>& S = state_of<R>(p);
    STP_CUDA(p, launch_path_targets<R>(geom_of<R>(p), S, S.tgt, p->stream));
    float h[STP_MLP_NTGT + 1];
    STP_CUDA(p, cudaMemcpyAsync(h, S.tgt, sizeof(h), cudaMemcpyDeviceToHost, p->stream));
    STP_CUDA(p, cudaStreamSynchronize(p->stream));
    if (h[STP_MLP_NTGT] == 0.f) return STP_NO_SOLUTION;
    std::memcpy(t, h, sizeof(float) * STP_MLP_NTGT);
    return STP_OK;
}

extern "C" stp_status stp_problem_targets(stp_problem* p, float* t) {
    clear_stale_error();
    if (!p || !t) return STP_ERR_INVALID;
    return p->precision == 0 ? targets_impl<float>(p, t) : targets_impl<double>(p, t);
}

extern "C" stp_status stp_problem_features(const stp_problem* p, float* x) {
    if (!p || !x) return STP_ERR_INVALID;
    double f[STP_MLP_IN] = {0};
    const int d = p->dof;
    for (int j = 0; j < d; ++j) {
        f[j] = 2.0 * (p->qs[j] - p->qlo[j]) / (p->qhi[j] - p->qlo[j]) - 1.0;
        f[7 + j] = 2.0 * (p->qg[j] - p->qlo[j]) / (p->qhi[j] - p->qlo[j]) - 1.0;
    }
    if (d == 2) f[14] = 1.0;
    else if (d == 6) f[15] = 1.0;
    else if (d == 7) f[16] = 1.0;
    if (p->M > 0) {
        double acc[7] = {0};
        for (int m = 0; m < p->M; ++m) {
            const double* w0 = &p->way[(size_t)m * p->K * 4];
            const double* w1 = &p->way[((size_t)m * p->K + p->K - 1) * 4];
            for (int i = 0; i < 3; ++i) {
                acc[i] += w0[1 + i];
                if (p->K > 1) acc[3 + i] += (w1[1 + i] - w0[1 + i]) / (w1[0] - w0[0]);
            }
            acc[6] += p->obs_r[m];
        }
        for (int i = 0; i < 7; ++i) f[17 + i] = acc[i] / p->M;
    }
    double D = 0.0;
    for (int j = 0; j < d; ++j) D += (p->qg[j] - p->qs[j]) * (p->qg[j] - p->qs[j]);
    D = std::sqrt(D);
    f[24] = p->prm.t_max / 60.0;
    f[25] = D / p->vmax / p->prm.t_max;
    for (int i = 0; i < STP_MLP_IN; ++i) x[i] = (float)f[i];
    return STP_OK;
}

// ---------------------------------------------------------------------------
// Failure-detection self-test: an mbarrier nobody arrives at, waited on with
// the library's bounded wait.
// ---------------------------------------------------------------------------
__global__ void k_wait_selftest(unsigned long long limit_ns, int* result) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    const unsigned long long t0 = global_ns();
    const bool ok = mbar_wait(&bar, 0, limit_ns);
    result[0] = ok ? 0 : 1;
    result[1] = (int)((global_ns() - t0) / 1000ull);  // microseconds waited
}

extern "C" stp_status stp_selftest_bounded_wait(unsigned long long limit_ns, int* waited_us) {
    clear_stale_error();
    if (limit_ns == 0 || limit_ns > 10000000000ull) return STP_ERR_INVALID;
    int* d = nullptr;
    int h[2] = {0, 0};
    cudaError_t e = cudaMalloc(&d, sizeof(h));
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaMalloc");
    k_wait_selftest<<<1, 32>>>(limit_ns, d);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "self-test kernel");
    if (waited_us) *waited_us = h[1];
    return h[0] ? STP_ERR_TIMEOUT : STP_OK;
}

static PersistArgs<float> batch_args(const stp_batch* b) {
    PersistArgs<float> a{};
    a.Gs = b->d_geom;
    a.Ss = b->d_state;
    a.max_iters = b->d_iters;
    a.P = (int)b->probs.size();
    a.team_size = b->team_ctas;
    a.sync = b->scratch.sync;
    a.queue = b->scratch.queue;
    a.team_prob = b->scratch.team_prob;
    a.abort_flag = b->scratch.abort_flag;
    return a;
}

extern "C" stp_status stp_batch_create(stp_problem* const* problems, int n, const stp_batch_params* bp,
                                       stp_batch** out) {
    clear_stale_error();
    if (!out || !problems || n < 1 || n > 65535) return STP_ERR_INVALID;
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (!problems[i] || problems[i]->precision != 0 || problems[i]->prm.continuous) return STP_ERR_INVALID;
    stp_batch* b = new (std::nothrow) stp_batch();
    if (!b) return STP_ERR_CUDA;
    b->probs.assign(problems, problems + n);
    b->iters_per_graph = bp && bp->iters_per_graph > 0 ? bp->iters_per_graph : 16;
    const int mode = bp ? bp->launch_mode : STP_LAUNCH_DEFAULT;
    if (mode < STP_LAUNCH_DEFAULT || mode > STP_LAUNCH_PERSISTENT || (bp && bp->team_ctas < 0)) {
        delete b;
        return STP_ERR_INVALID;
    }
    b->launch_mode = mode == STP_LAUNCH_STEPS ? 1 : 0;   // 0: persistent work queue, 1: per-step kernels
    b->team_ctas = bp && bp->team_ctas > 0 ? bp->team_ctas : 8;
    BatchShape& sh = b->shape;
    sh.P = n;
    sh.nn_ctas = bp && bp->nn_ctas > 0 ? bp->nn_ctas : 8;
    sh.validate_ctas = bp && bp->validate_ctas > 0 ? bp->validate_ctas : 2;
    std::vector<Geom<float>> hg(n);
    std::vector<State<float>> hs(n);
    std::vector<int> iters(n);
    int max_blob = 0;
    b->trivial.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        stp_problem* p = problems[i];
        bool same = true;
        for (int j = 0; j < p->dof; ++j) same = same && p->qs[j] == p->qg[j];
        b->trivial[i] = !p->start_free ? 1 : (same ? 2 : 0);
        hg[i] = p->gf;
        hs[i] = p->sf;
        b->traces.push_back(p->sf.trace);
        iters[i] = b->trivial[i] ? 0 : p->prm.max_iters;
        b->max_iters = std::max(b->max_iters, iters[i]);
        sh.max_W = std::max(sh.max_W, p->prm.ext_per_iter);
        sh.max_obs = std::max(sh.max_obs, p->M);
        max_blob = std::max(max_blob, (int)p->gf.blob_bytes);
    }
    sh.validate_smem = max_blob + (int)sizeof(int) * (2 * sh.max_W + 1);
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_geom, sizeof(Geom<float>) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_state, sizeof(State<float>) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_iters, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_geom, hg.data(), sizeof(Geom<float>) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_state, hs.data(), sizeof(State<float>) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_iters, iters.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
    if (e == cudaSuccess && b->launch_mode == 0) {
        // Persistent work queue: teams of team_ctas resident CTAs.
        b->persist_smem = persist_smem_bytes(max_blob, sh.max_W);
        int per_sm = 0;
        e = persist_blocks_per_sm<float>(7, b->persist_smem, &per_sm, persist_threads(true));
        if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
        if (e == cudaSuccess) {
            const int resident = validate_grid_blocks() * per_sm;
            b->team_ctas = std::min(b->team_ctas, resident);
            const int teams = std::max(1, std::min(resident / b->team_ctas, n));
            b->persist_grid = teams * b->team_ctas;
            b->scratch_bytes = persist_scratch_bytes(teams);
            e = cudaMalloc(&b->d_scratch, b->scratch_bytes);
        }
        if (e == cudaSuccess) {
            char* base = static_cast<char*>(b->d_scratch);
            const int teams = b->persist_grid / b->team_ctas;
            b->scratch.sync = reinterpret_cast<unsigned*>(base);
            b->scratch.queue = reinterpret_cast<int*>(base + sizeof(unsigned) * (size_t)teams * kPersistSyncStride);
            b->scratch.team_prob = b->scratch.queue + 1;
            b->scratch.abort_flag = b->scratch.queue + 1 + teams;
            // One graph: clear the scratch, then the persistent launch.
            cudaGraph_t g;
            PersistArgs<float> a = batch_args(b);
            cudaError_t ce = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
            cudaError_t le = cudaSuccess;
            if (ce == cudaSuccess) {
                le = cudaMemsetAsync(b->d_scratch, 0, b->scratch_bytes, b->stream);
                if (le == cudaSuccess)
                    le = launch_plan_persistent<float>(a, 7, b->persist_grid, b->persist_smem, b->stream,
                                                       persist_threads(true));
                cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
                if (le == cudaSuccess && ee == cudaSuccess) {
                    le = cudaGraphInstantiate(&b->graph, g, 0);
                    cudaGraphDestroy(g);
                } else if (ee == cudaSuccess) {
                    cudaGraphDestroy(g);
                }
            }
            if (ce != cudaSuccess || le != cudaSuccess || !b->graph) {
                // Not capturable here: plan with direct launches instead.
                (void)cudaGetLastError();
                b->graph = nullptr;
                b->graph_direct = true;
            }
        }
        if (e != cudaSuccess) {
            char buf[256];
            snprintf(buf, sizeof(buf), "stp_batch_create: %s", cudaGetErrorString(e));
            g_last_error = buf;
            stp_batch_free(b);
            return STP_ERR_CUDA;
        }
        b->ctl.resize(n);
        *out = b;
        return STP_OK;
    }
    if (e == cudaSuccess) {
        // Configure the batched collision kernel outside the capture.
        e = launch_validate_batch<float>(b->d_geom, b->d_state, 0, 0, sh.max_obs, 1, sh.validate_smem, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    }
    if (e == cudaSuccess) {
        cudaGraph_t g;
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        cudaError_t le = cudaSuccess;
        for (int i = 0; i < b->iters_per_graph && e == cudaSuccess && le == cudaSuccess; ++i)
            le = launch_iteration_batch<float>(b->d_geom, b->d_state, sh, b->stream);
        cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
        if (e == cudaSuccess) e = le != cudaSuccess ? le : ee;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
        if (ee == cudaSuccess) cudaGraphDestroy(g);
    }
    if (e != cudaSuccess) {
        char buf[256];
        snprintf(buf, sizeof(buf), "stp_batch_create: %s", cudaGetErrorString(e));
        g_last_error = buf;
        stp_batch_free(b);
        return STP_ERR_CUDA;
    }
    b->ctl.resize(n);
    *out = b;
    return STP_OK;
}

static bool hs_trace_matches(const stp_batch* b, int i) { return b->traces[i] == b->probs[i]->d_trace; }

extern "C" stp_status stp_batch_plan(stp_batch* b, stp_stats* stats, double* batch_ms) {
    clear_stale_error();
    if (!b) return STP_ERR_INVALID;
    const int n = (int)b->probs.size();
    for (int i = 0; i < n; ++i)
        if (b->probs[i]->prm.learned && !b->probs[i]->has_proposal) {
            b->last_error = "a learned member problem has no proposal (stp_set_proposal)";
            g_last_error = b->last_error;
            return STP_ERR_INVALID;
        }
    cudaStream_t st = b->stream;
    auto fail = [&](cudaError_t e, const char* where) {
        char buf[256];
        snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
        b->last_error = buf;
        g_last_error = buf;
        return STP_ERR_CUDA;
    };
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        stp_problem* p = b->probs[i];
        e = cudaMemsetAsync(p->sf.tile_cnt, 0, sizeof(int) * (size_t)(p->prm.n_roots + 1) * kMaxQTiles, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(p->sf.btile_cnt, 0, sizeof(int) * 2 * kMaxQTiles, st);
        // A member's trace is the one it had when the batch was created.
        if (e == cudaSuccess && p->d_trace && hs_trace_matches(b, i))
            e = cudaMemsetAsync(p->d_trace, 0xff,
                                sizeof(int) * (size_t)p->trace_iters * p->prm.ext_per_iter * kTraceInts, st);
    }
    if (e != cudaSuccess) return fail(e, "memset");
    if ((e = cudaEventRecord(b->ev0, st)) != cudaSuccess) return fail(e, "cudaEventRecord");
    if (b->launch_mode == 0) {
        // One persistent launch plans every problem (reset to path extraction).
        if (b->graph_direct) {
            if ((e = cudaMemsetAsync(b->d_scratch, 0, b->scratch_bytes, st)) != cudaSuccess) return fail(e, "memset");
            if ((e = launch_plan_persistent<float>(batch_args(b), 7, b->persist_grid, b->persist_smem, st,
                                                   persist_threads(true))) != cudaSuccess)
                return fail(e, "persistent launch");
        } else if ((e = cudaGraphLaunch(b->graph, st)) != cudaSuccess) {
            return fail(e, "cudaGraphLaunch");
        }
        if ((e = cudaEventRecord(b->ev1, st)) != cudaSuccess) return fail(e, "cudaEventRecord");
    } else {
        if ((e = launch_plan_reset_batch<float>(b->d_state, b->shape, b->d_iters, st)) != cudaSuccess)
            return fail(e, "reset");
        const int n_launch = (b->max_iters + b->iters_per_graph - 1) / b->iters_per_graph;
        for (int i = 0; i < n_launch; ++i)
            if ((e = cudaGraphLaunch(b->graph, st)) != cudaSuccess) return fail(e, "cudaGraphLaunch");
        if ((e = cudaEventRecord(b->ev1, st)) != cudaSuccess) return fail(e, "cudaEventRecord");
        if ((e = launch_extract_path_batch<float>(b->d_state, b->shape, st)) != cudaSuccess) return fail(e, "path");
    }
    for (int i = 0; i < n && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(&b->ctl[i], b->probs[i]->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(e, "readback");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b->ev0, b->ev1);
    if (batch_ms) *batch_ms = ms;
    stp_status result = STP_OK;
    // First solutions count from the start of the batch: the earliest start
    // of any problem (a queued problem starts when a team takes it).
    unsigned long long t0 = ~0ull;
    for (int i = 0; i < n; ++i)
        if (b->trivial[i] == 0) t0 = std::min(t0, b->ctl[i].t_start);
    for (int i = 0; i < n; ++i) {
        const Ctl& hc = b->ctl[i];
        stp_problem* p = b->probs[i];
        p->planned = b->trivial[i] == 0;
        stp_stats s;
        std::memset(&s, 0, sizeof(s));
        s.first_solution_iter = -1;
        s.first_solution_ms = -1.0;
        s.U = kInfD;
        s.C = kInfD;
        if (b->trivial[i] == 2) {
            s.U = 0.0;
            s.C = 0.0;
            s.first_solution_iter = 0;
            s.first_solution_ms = 0.0;
        } else if (b->trivial[i] == 0) {
            s.iterations = hc.iter;
            s.first_solution_iter = hc.first_iter;
            s.nodes = (long long)hc.st_ins;
            s.edges_validated = (long long)hc.st_ext;
            s.bridges_validated = (long long)hc.st_bridge;
            s.root_checks = (long long)hc.st_root;
            s.check_points = (long long)hc.st_points;
            s.pair_tests = (long long)hc.st_pairs;
            s.nn_evals = (long long)hc.st_nn_evals;
            s.nn_nodes = (long long)hc.st_nn_nodes;
            s.bridge_evals = (long long)hc.st_br_evals;
            s.bridge_nodes = (long long)hc.st_br_nodes;
            s.first_solution_ms = hc.first_iter >= 0 ? (double)(hc.t_first - t0) * 1e-6 : -1.0;
            s.plan_ms = hc.t_end > hc.t_start ? (double)(hc.t_end - hc.t_start) * 1e-6 : ms;
            s.U = hc.U;
            s.C = hc.C;
            if (hc.err & kErrCapacity) result = STP_ERR_CAPACITY;
            if ((hc.err & kErrTimeout) && result == STP_OK) result = STP_ERR_TIMEOUT;
        }
        if (stats) stats[i] = s;
    }
    return result;
}

extern "C" stp_status stp_batch_path(stp_batch* b, int i, double* path, int cap, int* n_path) {
    if (!b || i < 0 || i >= (int)b->probs.size() || !n_path) return STP_ERR_INVALID;
    stp_problem* p = b->probs[i];
    *n_path = 0;
    if (b->trivial[i] == 2) {
        *n_path = 1;
        if (path) {
            if (cap < 1) return STP_ERR_CAPACITY;
            for (int j = 0; j < p->dof; ++j) path[j] = p->qs[j];
            path[p->dof] = 0.0;
        }
        return STP_OK;
    }
    if (b->trivial[i] == 1) return STP_OK;
    int len = 0;
    STP_CUDA(p, cudaMemcpy(&len, p->sf.path_len, sizeof(int), cudaMemcpyDeviceToHost));
    if (len < 0) return STP_ERR_CAPACITY;
    *n_path = len;
    if (path && len > 0) return copy_path<float>(p, len, path, cap);
    return STP_OK;
}

extern "C" void stp_batch_free(stp_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->d_scratch) cudaFree(b->d_scratch);
    if (b->d_geom) cudaFree(b->d_geom);
    if (b->d_state) cudaFree(b->d_state);
    if (b->d_iters) cudaFree(b->d_iters);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}
