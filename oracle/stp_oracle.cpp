// ST-pRRTC oracle: plain, slow, single-threaded FP64 CPU restatement of the
// batch-synchronous space-time Extend loop (Sec. "Space-Time pRRTC": interval
// root, Algorithms 1-2, Eqs. goal-time-lower-bound, conditional-query-time,
// space-time-metric; Sec. "Practical Root Recycling": Algorithm 3,
// Eq. max-speed-extension; problem model of Sec. "Problem Formulation").
//
// TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
// CPU-baseline leg may load this library. It shares no code, header, table or
// constant with the CUDA path; the CUDA library must never call it.
//
// Floating point is double throughout. The file is compiled with
// -ffp-contract=off so that x86 and Arm hosts round identically.
//
// Readings of points the paper leaves open are marked "Reading:" in comments.
// Philox4x32-10 follows its published definition (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11).
//
// Parity status: every function here is pinned by tests/test_oracle_*.py
// (worked examples of Figs. interval-root and method, closed forms, brute force,
// invariants); the per-worker decisions (direction, group, new-root coin,
// conditional query time, NN parents, bridge rank, improvement test, publish
// order, round-robin slots) are re-derived by brute force from the decision
// records and by hand cases in tests/test_oracle_decisions.py. End-to-end
// success rates and arrival values of the synthetic workloads are parity
// unpinned (the paper's suites are not available).
//
// Every run records one decision record per worker and iteration (the layout
// the device library's trace writes too). Follow mode takes a device run's
// records: where an FP64 margin is below the flag threshold the oracle adopts
// the device's choice, elsewhere any difference is reported.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <vector>

namespace {

const double kInf = std::numeric_limits<double>::infinity();

// ---------------------------------------------------------------------------
// Philox4x32-10 (SC'11). Counter (c0,c1,c2,c3), key (k0,k1).
// ---------------------------------------------------------------------------
const uint32_t kPhiloxM0 = 0xD2511F53u;
const uint32_t kPhiloxM1 = 0xCD9E8D57u;
const uint32_t kPhiloxW0 = 0x9E3779B9u;
const uint32_t kPhiloxW1 = 0xBB67AE85u;

void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += kPhiloxW0;
            k1 += kPhiloxW1;
        }
        uint64_t p0 = (uint64_t)kPhiloxM0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)kPhiloxM1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
    for (int i = 0; i < 4; ++i) out[i] = c[i];
}

// Reading (RNG unnamed in the paper): per (problem p, iteration k, worker w)
// the draws are slots s = 0,1,2,...: slot s is word s%4 of the Philox block with
// counter (s/4, w, k, p) and key (seed lo, seed hi).
// Slot map: 0 group, 1 guided coin, 2 T position, 3 new-root coin,
// 4..4+d-1 configuration sample q_r, 4+d query time t_r; the learned branch
// adds 12 learned coin, 13 waypoint index, 14 mixture component, 15-16
// Box-Muller uniforms.
struct Draws {
    uint32_t raw[20];
    void fill(uint64_t seed, uint32_t problem, uint32_t iter, uint32_t worker, int nslots) {
        uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        for (int b = 0; b * 4 < nslots; ++b) {
            uint32_t ctr[4] = {(uint32_t)b, worker, iter, problem};
            philox4x32_10(ctr, key, &raw[4 * b]);
        }
    }
    // u = (x >> 8) * 2^-24, exactly representable in single and double.
    double u(int slot) const { return (double)(raw[slot] >> 8) * (1.0 / 16777216.0); }
    // group index floor(u * N) evaluated exactly in integers.
    int group(int slot, int n) const {
        return (int)(((uint64_t)(raw[slot] >> 8) * (uint64_t)n) >> 24);
    }
};

// ---------------------------------------------------------------------------
// Problem model (Sec. "Problem Formulation"): C subset of R^d with Euclidean
// metric, velocity bound v_max, horizon [0,H], known obstacle trajectories.
// ---------------------------------------------------------------------------
struct Problem {
    int dof = 0;
    bool arm = false;              // false: point robot (translation only)
    std::vector<double> dh;        // [dof][4] a, alpha, d, theta0 (standard DH)
    std::vector<double> qlo, qhi;  // [dof]
    std::vector<int> sph_link;     // [S] frame index 0..dof
    std::vector<double> sph_p;     // [S][3] local centre
    std::vector<double> sph_r;     // [S]
    double vmax = 1.0;
    int n_obs = 0, n_way = 0;
    std::vector<double> obs_r;     // [M]
    std::vector<double> way;       // [M][K][4] t, x, y, z
    std::vector<double> qs, qg;    // [dof]
    // Self-collision (arms, optional): sphere pairs (i < j) on frames at least
    // two apart that do not already overlap at q = 0.
    std::vector<std::pair<int, int>> self_pairs;
};

double dist(const double* a, const double* b, int d) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        double e = b[j] - a[j];
        s += e * e;
    }
    return std::sqrt(s);
}

// A rigid frame: rotation R (row-major 3x3) and origin o.
struct Frame {
    double R[9];
    double o[3];
};

// Standard DH link transform A = Rz(theta) Tz(d) Tx(a) Rx(alpha).
Frame dh_transform(double a, double alpha, double d, double theta) {
    double ct = std::cos(theta), st = std::sin(theta);
    double ca = std::cos(alpha), sa = std::sin(alpha);
    Frame f;
    f.R[0] = ct; f.R[1] = -st * ca; f.R[2] = st * sa;
    f.R[3] = st; f.R[4] = ct * ca;  f.R[5] = -ct * sa;
    f.R[6] = 0;  f.R[7] = sa;       f.R[8] = ca;
    f.o[0] = a * ct;
    f.o[1] = a * st;
    f.o[2] = d;
    return f;
}

Frame compose(const Frame& A, const Frame& B) {
    Frame C;
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A.R[3 * i + k] * B.R[3 * k + j];
            C.R[3 * i + j] = s;
        }
        double s = A.o[i];
        for (int k = 0; k < 3; ++k) s += A.R[3 * i + k] * B.o[k];
        C.o[i] = s;
    }
    return C;
}

// Frames 0..dof. Frame 0 is the base. For the point robot, frame 0 is the
// identity rotation placed at (q0, q1, q2) (missing coordinates are 0) and the
// configuration is a position in the plane or space.
void forward_kinematics(const Problem& P, const double* q, std::vector<Frame>& frames) {
    Frame base;
    for (int i = 0; i < 9; ++i) base.R[i] = (i % 4 == 0) ? 1.0 : 0.0;
    base.o[0] = base.o[1] = base.o[2] = 0.0;
    frames.assign(1, base);
    if (!P.arm) {
        for (int j = 0; j < 3 && j < P.dof; ++j) frames[0].o[j] = q[j];
        return;
    }
    for (int j = 0; j < P.dof; ++j) {
        const double* row = &P.dh[4 * j];
        Frame A = dh_transform(row[0], row[1], row[2], row[3] + q[j]);
        frames.push_back(compose(frames.back(), A));
    }
}

void sphere_centres(const Problem& P, const std::vector<Frame>& frames, std::vector<double>& c) {
    int S = (int)P.sph_r.size();
    c.assign(3 * S, 0.0);
    for (int s = 0; s < S; ++s) {
        const Frame& F = frames[P.sph_link[s]];
        const double* p = &P.sph_p[3 * s];
        for (int i = 0; i < 3; ++i) {
            double v = F.o[i];
            for (int k = 0; k < 3; ++k) v += F.R[3 * i + k] * p[k];
            c[3 * s + i] = v;
        }
    }
}

// Obstacle position at absolute time t: piecewise-linear interpolation of the
// waypoints (Sec. "Simulation Protocol": positions interpolated at each
// absolute query time). Reading: before the first / after the last waypoint the
// obstacle holds that waypoint.
void obstacle_position(const Problem& P, int m, double t, double out[3]) {
    const double* W = &P.way[(size_t)m * P.n_way * 4];
    int K = P.n_way;
    if (t <= W[0]) {
        for (int i = 0; i < 3; ++i) out[i] = W[1 + i];
        return;
    }
    if (t >= W[4 * (K - 1)]) {
        for (int i = 0; i < 3; ++i) out[i] = W[4 * (K - 1) + 1 + i];
        return;
    }
    int k = 0;
    while (!(t < W[4 * (k + 1)])) ++k;  // W[4k] <= t < W[4(k+1)]
    double t0 = W[4 * k], t1 = W[4 * (k + 1)];
    double f = (t - t0) / (t1 - t0);
    for (int i = 0; i < 3; ++i) {
        double a = W[4 * k + 1 + i], b = W[4 * (k + 1) + 1 + i];
        out[i] = a + f * (b - a);
    }
}

bool in_bounds(const Problem& P, const double* q) {
    for (int j = 0; j < P.dof; ++j)
        if (q[j] < P.qlo[j] || q[j] > P.qhi[j]) return false;
    return true;
}

// Clearance of state (q,t): min over sphere pairs of |p - o| - r - r_o.
// Reading (collision predicate): a pair collides iff |p-o|^2 < (r+r_o)^2;
// touching is free; a configuration outside the bounds collides.
// Returns true iff collision-free.
bool state_free(const Problem& P, const double* q, double t, double* clearance) {
    std::vector<Frame> frames;
    std::vector<double> c;
    forward_kinematics(P, q, frames);
    sphere_centres(P, frames, c);
    bool free = in_bounds(P, q);
    double clr = kInf;
    int S = (int)P.sph_r.size();
    // Self-collision: the same predicate between the robot's own spheres.
    for (const auto& pr : P.self_pairs) {
        const int a = pr.first, b = pr.second;
        double dx = c[3 * a] - c[3 * b], dy = c[3 * a + 1] - c[3 * b + 1], dz = c[3 * a + 2] - c[3 * b + 2];
        double d2 = dx * dx + dy * dy + dz * dz;
        double rr = P.sph_r[a] + P.sph_r[b];
        if (d2 < rr * rr) free = false;
        double cl = std::sqrt(d2) - rr;
        if (cl < clr) clr = cl;
    }
    for (int m = 0; m < P.n_obs; ++m) {
        double o[3];
        obstacle_position(P, m, t, o);
        for (int s = 0; s < S; ++s) {
            double dx = c[3 * s] - o[0], dy = c[3 * s + 1] - o[1], dz = c[3 * s + 2] - o[2];
            double d2 = dx * dx + dy * dy + dz * dz;
            double rr = P.sph_r[s] + P.obs_r[m];
            if (d2 < rr * rr) free = false;
            double cl = std::sqrt(d2) - rr;
            if (cl < clr) clr = cl;
        }
    }
    if (clearance) *clearance = clr;
    return free;
}

// Reading (edge resolution): an edge (q_a,t_a)->(q_b,t_b) is checked at
// c = max(1, ceil(max(D, v_max |t_b - t_a|) / res - 1e-3)) points s_j = j/c,
// j = 1..c (the start state was validated when it was inserted). The 1e-3
// slack lets the spacing exceed res by at most 0.1 % of a step and makes c
// insensitive to rounding when the length is an exact multiple of res (every
// root-recycling step of length eta is one).
int edge_check_count(const Problem& P, const double* qa, double ta, const double* qb, double tb,
                     double res, double* int_margin) {
    double D = dist(qa, qb, P.dof);
    double L = std::max(D, P.vmax * std::fabs(tb - ta));
    double x = L / res - 1e-3;
    double c = std::ceil(x);
    if (int_margin) {
        double fr = x - std::floor(x);
        *int_margin = std::min(fr, 1.0 - fr);
    }
    return std::max(1, (int)c);
}

// Edge verdict with its FP64 clearance (min over all check points, no early
// exit) and check-point count.
// bound_margin: min over check points and joints of (q - lo, hi - q), the
// signed distance of the checked states from the configuration-box boundary.
// force_count > 0 checks that many points instead (follow mode adopts a
// reduced-precision run's count where the rounding of c is undecided).
bool edge_free(const Problem& P, const double* qa, double ta, const double* qb, double tb, double res,
               double* clearance, int* nchk, double* int_margin, double* bound_margin = nullptr,
               int force_count = 0) {
    int c = edge_check_count(P, qa, ta, qb, tb, res, int_margin);
    if (force_count > 0) c = force_count;
    bool free = true;
    double clr = kInf, bm = kInf;
    std::vector<double> q(P.dof);
    for (int j = 1; j <= c; ++j) {
        double s = (double)j / (double)c;
        for (int i = 0; i < P.dof; ++i) {
            q[i] = qa[i] + s * (qb[i] - qa[i]);
            bm = std::min(bm, std::min(q[i] - P.qlo[i], P.qhi[i] - q[i]));
        }
        double t = ta + s * (tb - ta);
        double cl;
        if (!state_free(P, q.data(), t, &cl)) free = false;
        if (cl < clr) clr = cl;
    }
    if (clearance) *clearance = clr;
    if (nchk) *nchk = c;
    if (bound_margin) *bound_margin = bm;
    return free;
}

// Continuous edge validation for a point robot (translation only): between
// consecutive breakpoints (the edge's end times and every obstacle waypoint
// time inside them) each robot sphere and each obstacle move linearly, so
// their difference d(t) runs along the segment from d(tau_i) to d(tau_i+1) and
// its smallest norm is the distance from the origin to that segment (closed
// form). Clearance = the exact minimum of |p - o| - r - r_o over [t_a, t_b];
// a pair collides iff that minimum squared distance < (r + r_o)^2 (touching is
// free); the segment stays in the convex configuration box iff both ends do.
bool edge_free_continuous(const Problem& P, const double* qa, double ta, const double* qb, double tb,
                          double* clearance) {
    const int S = (int)P.sph_r.size();
    bool free = in_bounds(P, qa) && in_bounds(P, qb);
    double clr = kInf;
    std::vector<Frame> fa, fb;
    std::vector<double> ca, cb, qm(P.dof);
    for (int m = 0; m < P.n_obs; ++m) {
        const double* W = &P.way[(size_t)m * P.n_way * 4];
        std::vector<double> tau{ta};
        for (int k = 0; k < P.n_way; ++k)
            if (W[4 * k] > ta && W[4 * k] < tb) tau.push_back(W[4 * k]);
        tau.push_back(tb);
        for (size_t i = 0; i + 1 < tau.size(); ++i) {
            const double t0 = tau[i], t1 = tau[i + 1];
            const double f0 = tb > ta ? (t0 - ta) / (tb - ta) : 0.0;
            const double f1 = tb > ta ? (t1 - ta) / (tb - ta) : 0.0;
            for (int j = 0; j < P.dof; ++j) qm[j] = qa[j] + f0 * (qb[j] - qa[j]);
            forward_kinematics(P, qm.data(), fa);
            sphere_centres(P, fa, ca);
            for (int j = 0; j < P.dof; ++j) qm[j] = qa[j] + f1 * (qb[j] - qa[j]);
            forward_kinematics(P, qm.data(), fb);
            sphere_centres(P, fb, cb);
            double o0[3], o1[3];
            obstacle_position(P, m, t0, o0);
            obstacle_position(P, m, t1, o1);
            for (int sp = 0; sp < S; ++sp) {
                double d0[3], w[3];
                for (int k = 0; k < 3; ++k) {
                    d0[k] = ca[3 * sp + k] - o0[k];
                    w[k] = (cb[3 * sp + k] - o1[k]) - d0[k];
                }
                const double a = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
                const double b = d0[0] * w[0] + d0[1] * w[1] + d0[2] * w[2];
                double u = a > 0.0 ? -b / a : 0.0;
                u = std::min(std::max(u, 0.0), 1.0);
                double d2 = 0.0;
                for (int k = 0; k < 3; ++k) {
                    const double e = d0[k] + u * w[k];
                    d2 += e * e;
                }
                const double rr = P.sph_r[sp] + P.obs_r[m];
                if (d2 < rr * rr) free = false;
                clr = std::min(clr, std::sqrt(d2) - rr);
            }
        }
    }
    if (clearance) *clearance = clr;
    return free;
}

// ---------------------------------------------------------------------------
// Goal-time grid (Eq. goal-time-lower-bound): L_g = D(q_s,q_g)/v_max,
// k_min = ceil(L_g/dt); goal checks at k dt in [L_g, H].
// ---------------------------------------------------------------------------
struct GoalGrid {
    double Lg = 0, dt = 0, H = 0;
    long kmin = 0, kmax = 0;        // checks k = kmin..kmax (k dt <= H)
    std::vector<char> free;         // [kmax - kmin + 1]
    std::vector<double> clearance;  // [kmax - kmin + 1]
    bool is_free(long k) const {
        if (k < kmin || k > kmax) return false;
        return free[k - kmin] != 0;
    }
};

void build_goal_grid(const Problem& P, double H, double dt, GoalGrid& G) {
    G.Lg = dist(P.qs.data(), P.qg.data(), P.dof) / P.vmax;
    G.dt = dt;
    G.H = H;
    G.kmin = (long)std::ceil(G.Lg / dt);
    G.kmax = (long)std::floor(H / dt);
    long n = G.kmax - G.kmin + 1;
    if (n < 0) n = 0;
    G.free.assign(n, 0);
    G.clearance.assign(n, 0.0);
    for (long i = 0; i < n; ++i) {
        double t = (double)(G.kmin + i) * dt;
        double cl;
        G.free[i] = state_free(P, P.qg.data(), t, &cl) ? 1 : 0;
        G.clearance[i] = cl;
    }
}

// ---------------------------------------------------------------------------
// Interval-root allocation (Sec. "Interval Root").
// ---------------------------------------------------------------------------
struct Piece {
    double lo, hi;
    int group;
};

struct IntervalAlloc {
    double Lg = 0, H = 0, dt = 0;
    int N = 0;
    std::vector<std::pair<double, double>> windows;  // guided windows in [L_g, H]
    double Ubar = 0, width = 0;                      // uniform interval width
    std::vector<Piece> pieces;                       // time order
    std::vector<std::vector<int>> group_pieces;      // indices into pieces
    std::vector<double> group_measure;
};

// A goal check k that finds (q_g, k dt) free contributes the window
// [k dt - dt/2, k dt + dt/2], cut to [L_g, H]; windows that touch are joined,
// and the joined windows are the guided windows.
void build_windows(IntervalAlloc& A, long kmin, long kmax, const char* free_flags) {
    A.windows.clear();
    long k = kmin;
    while (k <= kmax) {
        if (!free_flags[k - kmin]) {
            ++k;
            continue;
        }
        long k0 = k;
        while (k + 1 <= kmax && free_flags[k + 1 - kmin]) ++k;
        double lo = (double)k0 * A.dt - 0.5 * A.dt;
        double hi = (double)k * A.dt + 0.5 * A.dt;
        lo = std::max(lo, A.Lg);
        hi = std::min(hi, A.H);
        if (hi > lo) A.windows.push_back({lo, hi});
        ++k;
    }
}

// With Ubar = min(H, U): N equal uniform intervals on [L_g, Ubar); the guided
// windows below Ubar are concatenated in time order (gaps skipped) and group g
// receives the measure in [g G/N, (g+1) G/N) of the concatenation.
void partition(IntervalAlloc& A, double U) {
    A.Ubar = std::min(A.H, U);
    A.width = (A.Ubar - A.Lg) / (double)A.N;
    A.pieces.clear();
    A.group_pieces.assign(A.N, {});
    A.group_measure.assign(A.N, 0.0);
    std::vector<std::pair<double, double>> clipped;
    for (auto& w : A.windows) {
        if (w.first >= A.Ubar) continue;
        double hi = std::min(w.second, A.Ubar);
        if (hi > w.first) clipped.push_back({w.first, hi});
    }
    std::vector<double> start_measure(clipped.size());
    double G = 0.0;
    for (size_t i = 0; i < clipped.size(); ++i) {
        start_measure[i] = G;
        G += clipped[i].second - clipped[i].first;
    }
    if (G <= 0.0) return;
    for (int g = 0; g < A.N; ++g) {
        double mlo = G * (double)g / (double)A.N;
        double mhi = (g == A.N - 1) ? G : G * (double)(g + 1) / (double)A.N;
        for (size_t i = 0; i < clipped.size(); ++i) {
            double m0 = start_measure[i];
            double m1 = (i + 1 < clipped.size()) ? start_measure[i + 1] : G;
            double a = std::max(mlo, m0), b = std::min(mhi, m1);
            if (b > a) {
                Piece p;
                p.lo = clipped[i].first + (a - m0);
                p.hi = clipped[i].first + (b - m0);
                p.group = g;
                A.group_pieces[g].push_back((int)A.pieces.size());
                A.pieces.push_back(p);
                A.group_measure[g] += p.hi - p.lo;
            }
        }
    }
}

// Group i draws T, with probability p_guided, from the guided pieces of its
// interval (the uniform interval when there are none), otherwise uniformly
// from I_i.
// walk_margin (optional): the smallest |p - len| met while walking the
// pieces (where a rounding of p would move T across a gap between pieces).
double sample_goal_time(const IntervalAlloc& A, int g, double u_coin, double u_pos, double p_guided,
                        bool* guided, double* walk_margin = nullptr) {
    if (walk_margin) *walk_margin = kInf;
    if (u_coin < p_guided && A.group_measure[g] > 0.0) {
        *guided = true;
        double p = u_pos * A.group_measure[g];
        const std::vector<int>& idx = A.group_pieces[g];
        for (size_t j = 0; j < idx.size(); ++j) {
            const Piece& pc = A.pieces[idx[j]];
            double len = pc.hi - pc.lo;
            if (walk_margin && j + 1 < idx.size()) *walk_margin = std::min(*walk_margin, std::fabs(p - len));
            if (p < len || j + 1 == idx.size()) return std::min(pc.lo + p, pc.hi);
            p -= len;
        }
    }
    *guided = false;
    double lo = A.Lg + (double)g * A.width;
    return lo + u_pos * A.width;
}

// ---------------------------------------------------------------------------
// Planner state.
// ---------------------------------------------------------------------------
struct Node {
    std::vector<double> q;
    double t;
    int parent;    // index in the same arena, -1 for a root
    double troot;  // backward: root (arrival) time of the tree; forward: 0
    double cost;   // configuration-space path length to the tree root
    int tree;      // interval root: backward tree id; root recycling: slot generation
    int iter;      // iteration that inserted the node (-1: initial roots)
};

struct Tree {  // interval-root backward tree
    int group;
    double T;
};

struct Slot {  // root-recycling slot
    bool has_root = false;
    bool active = false;
    double T = kInf;
    long k = -1;  // grid index of T (T = k dt)
    int gen = 0;
};

// Root recycling on an incumbent decrease (Algorithm 3): roots with T_i >= U
// become inactive; slots with T_i > U (and empty slots) are donors. Reading
// (replacement placement): with K_U grid indices in [L_grid, U) and m donors
// in slot order, donor j targets index kmin + floor((2j+1) K_U / (2m)) and
// scans outward, below first, for a free goal check not held by an active root.
// A donor without a candidate stays inactive. Returns the replaced slots.
template <class IsFree>
std::vector<int> recycle_rule(std::vector<Slot>& slots, double U, long kmin, double dt, IsFree is_free) {
    long kU = kmin;
    while ((double)kU * dt < U) ++kU;  // first index with k dt >= U
    std::vector<long> held;
    std::vector<int> donors, replaced;
    for (size_t i = 0; i < slots.size(); ++i) {
        Slot& s = slots[i];
        if (s.has_root && s.T >= U) s.active = false;
        if (!s.has_root || s.T > U) donors.push_back((int)i);
        if (s.has_root && s.active) held.push_back(s.k);
    }
    int m = (int)donors.size();
    long KU = kU - kmin;
    for (int j = 0; j < m && KU > 0; ++j) {
        long target = kmin + ((2L * j + 1) * KU) / (2L * m);
        long found = -1;
        for (long o = 0; o < KU && found < 0; ++o) {
            long cand[2] = {target - o, target + o};
            for (int c = 0; c < (o == 0 ? 1 : 2); ++c) {
                long k = cand[c];
                if (k < kmin || k >= kU) continue;
                if (!is_free(k)) continue;
                if (std::find(held.begin(), held.end(), k) != held.end()) continue;
                found = k;
                break;
            }
        }
        if (found < 0) continue;
        Slot& s = slots[donors[j]];
        s.has_root = true;
        s.active = true;
        s.k = found;
        s.T = (double)found * dt;
        s.gen += 1;
        held.push_back(found);
        replaced.push_back(donors[j]);
    }
    return replaced;
}

// ---------------------------------------------------------------------------
// Learned sampling branch (the method's GPU form: a learned proposal with 10 %
// plain samples). A network output y[160] gives a mixture of 8 Gaussians over
// tau = T/H (logits y[0:8], means y[8:16], log standard deviations y[16:24]
// clamped to [-7, 2]) and 16 waypoints as offsets y[24 + 8 i + j] from the
// straight line: waypoint i, joint j, in coordinates normalised to [-1, 1]
// over the joint box, is the offset plus (1 - f_i) u_s + f_i u_g with
// f_i = (i + 1) / 17 and u_s, u_g the normalised start and goal, clipped to
// [-1, 1]. Readings: a worker is learned when its coin
// (slot 12) is below p_learned = 0.9 (integer threshold ceil(0.9 2^24)); it
// then draws q_r uniformly in +-0.1 of each joint's range around waypoint i
// (slot 13, uniform over the 16), clipped to C, reusing the plain q_r
// uniforms; in interval root it also draws T from the mixture (component by
// slot 14, Box-Muller normal from slots 15-16) and keeps it only when it lies
// in the sampled group's uniform interval, otherwise the plain T stands.
// ---------------------------------------------------------------------------
constexpr uint32_t kThrLearned = 15099495u;  // ceil(0.9 * 2^24)
constexpr double kLearnedHalfWidth = 0.1;    // fraction of each joint range

struct Learned {
    bool on = false;
    double cw[8] = {0}, mu[8] = {0}, sig[8] = {0};  // cumulative weights; T mean / sd in seconds
    std::vector<double> wq;                          // [16][dof]
};

void build_learned(Learned& L, const double* y, const std::vector<double>& lo, const std::vector<double>& hi,
                   const std::vector<double>& qs, const std::vector<double>& qg, int dof, double H) {
    L.on = true;
    double amax = y[0];
    for (int k = 1; k < 8; ++k) amax = std::max(amax, y[k]);
    double e[8], tot = 0.0;
    for (int k = 0; k < 8; ++k) {
        e[k] = std::exp(y[k] - amax);
        tot += e[k];
    }
    double acc = 0.0;
    for (int k = 0; k < 8; ++k) {
        acc += e[k];
        L.cw[k] = acc / tot;
    }
    L.cw[7] = 1.0;
    for (int k = 0; k < 8; ++k) {
        L.mu[k] = y[8 + k] * H;
        L.sig[k] = std::exp(std::min(std::max(y[16 + k], -7.0), 2.0)) * H;
    }
    L.wq.assign(16 * (size_t)dof, 0.0);
    for (int i = 0; i < 16; ++i) {
        const double f = (double)(i + 1) / 17.0;
        for (int j = 0; j < dof; ++j) {
            const double us = 2.0 * (qs[j] - lo[j]) / (hi[j] - lo[j]) - 1.0;
            const double ug = 2.0 * (qg[j] - lo[j]) / (hi[j] - lo[j]) - 1.0;
            double u = y[24 + 8 * i + j] + ((1.0 - f) * us + f * ug);
            u = std::min(std::max(u, -1.0), 1.0);
            L.wq[(size_t)i * dof + j] = lo[j] + (u + 1.0) * 0.5 * (hi[j] - lo[j]);
        }
    }
}

// q_r of a learned worker (overwrites qr); margins of the clip tests are noted.
void learned_q(const Learned& L, const Draws& dr, const std::vector<double>& lo, const std::vector<double>& hi,
               int dof, double* qr) {
    const int i = dr.group(13, 16);
    for (int j = 0; j < dof; ++j) {
        const double half = kLearnedHalfWidth * (hi[j] - lo[j]);
        double q = L.wq[(size_t)i * dof + j] + half * (2.0 * dr.u(4 + j) - 1.0);
        qr[j] = std::min(std::max(q, lo[j]), hi[j]);
    }
}

// Mixture goal time of a learned worker; returns the component's draw.
double learned_T(const Learned& L, const Draws& dr, double* comp_margin) {
    const double u = dr.u(14);
    int k = 0;
    while (k < 7 && !(u < L.cw[k])) ++k;
    double m = std::fabs(L.cw[k] - u);
    if (k > 0) m = std::min(m, std::fabs(u - L.cw[k - 1]));
    *comp_margin = m;
    const double u1 = 1.0 - dr.u(15), u2 = dr.u(16);
    const double z = std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586476925 * u2);
    return L.mu[k] + L.sig[k] * z;
}

struct Params {
    int variant = 0;  // 0 interval root, 1 root recycling, 2 no recycling (fixed forest)
    int N = 4;
    int W = 64;
    int max_iters = 100;
    double eta = 0.1, res = 0.01, dt = 0.02, p_new = 0.05, p_guided = 0.95, H = 10.0;
    uint64_t seed = 0;
    uint32_t problem_id = 0;
    // Margin below which a decision is flagged as rounding-sensitive. FP32 runs
    // carry coordinate errors up to a few 1e-6 (steering accumulates about
    // eps |q| / alpha per tree level), so 1e-5 keeps a safety factor above it.
    double flag_tol = 1e-5;
    double flag_clear = 1e-5;  // clearance band (m)
    const double* proposal = nullptr;  // learned branch: network output y[160], or none
    int continuous = 0;                // point robots: closed-form edge validation
    // Follow mode (parity of a reduced-precision run, see struct Follow):
    // decision records [follow_iters][W][kTraceInts] and goal-grid free flags
    // [follow_nk] of that run, or none.
    const int* follow_rec = nullptr;
    int follow_iters = 0;
    const unsigned char* follow_grid = nullptr;
    int follow_nk = 0;
};

// Decision record of one worker in one iteration. The same field meanings are
// written, independently, by the device library's trace (an interface, not
// shared code): the oracle records its own decisions here, and in follow mode
// it reads the device's.
//   [0] flags (TraceFlag), [1] group (interval) / slot (recycling) or -1,
//   [2] NN parent index (-1: virtual root or none), [3] extension check count
//   (0: no edge), [4] bridge candidate arena (-1 forward tree, else backward
//   group / slot), [5] bridge candidate index (-1), [6] bridge check count,
//   [7] inserted node index (-1), [8] learned mixture component (-1),
//   [9] the goal time T as float bits (interval root; 0 otherwise).
constexpr int kTraceInts = 10;
enum TraceFlag {
    kTrFwd = 1,          // forward worker: (w + k) even
    kTrSampled = 2,      // interval: non-empty query-time window; recycling: a source tree
    kTrVirtual = 4,      // backward source is a new (virtual) root
    kTrEmit = 8,         // extension edge steered and inside the horizon
    kTrRootHit = 16,     // the sampled goal root collides
    kTrExtHit = 32,      // the extension edge collides
    kTrInserted = 64,
    kTrBrCand = 128,     // an admissible bridge candidate exists
    kTrBrEmit = 256,     // the candidate would improve (U, C) and is validated
    kTrBrHit = 512,      // the bridge edge collides
    kTrWinner = 1024,    // this worker's bridge is the iteration's published solution
    kTrLearned = 2048,   // learned worker (slot-12 coin)
    kTrLearnedT = 4096,  // goal time taken from the mixture
    kTrGuided = 8192,    // goal time drawn from the group's guided pieces
};
// Decision kinds counted in follow mode.
enum Kind {
    kKDirection, kKGroup, kKLearnedComp, kKLearnedT, kKRoot, kKWindow, kKVirtual, kKParent, kKEmit,
    kKExtCount, kKExtHit, kKInserted, kKBrCand, kKBrEmit, kKBrCount, kKBrHit, kKWinner, kKGrid, kKGuided,
    kKGoalTime, kKinds
};

// Smallest decision margins seen during one iteration (test diagnostics for
// comparing a reduced-precision run with this FP64 one). Trees depend on NN
// choices, admissibility, check counts, interval emptiness, horizon and box
// boundaries, bridge ranks (which edge is tested and so which U is found) and
// clearances; comparisons of path length C alone only choose between
// solutions of equal U and never change a tree, so they are kept apart.
struct Margin {
    double nn = kInf, clearance = kInf, count = kInf, interval = kInf, bounds = kInf, rank = kInf;
    double cost = kInf;
    double min_all() const {
        return std::min(std::min(std::min(nn, count), std::min(interval, bounds)), rank);
    }
};

struct Result {
    int dof = 0, N = 0, variant = 0;
    std::vector<Node> fwd;
    std::vector<std::vector<Node>> seg;
    std::vector<Tree> trees;
    std::vector<Slot> slots;
    double U = kInf, C = kInf;
    int inc_fwd = -1, inc_seg = -1, inc_bwd = -1;
    int iters = 0, first_iter = -1;
    long long ext_checked = 0, bridge_checked = 0, root_checked = 0, inserted = 0;
    std::vector<double> path;  // [len][dof+1]
    std::vector<double> U_hist, C_hist, margin_hist, clear_hist;
    std::vector<double> margin_types;  // [iters][6]: nn, count, interval, bounds, rank, clearance
    int status = 0;  // 0 solved, 5 no solution
    std::vector<double> goal_clearance;
    long goal_kmin = 0;
    // Decision records [iters][W][kTraceInts] and per worker (T, t_r, window
    // lo, window hi) [iters][W][4] (NaN where not drawn).
    std::vector<int> trace;
    std::vector<double> trace_d;
    // Follow mode: decisions adopted from the device run per kind, those where
    // its choice differed, and unflagged differences as (iter, worker, kind).
    long long followed[kKinds] = {}, flagged_diff[kKinds] = {};
    std::vector<int> unflagged;
};

struct Proposal {
    bool ok = false;
    bool forward = true;
    int seg = -1;           // group (interval) or slot (recycling)
    int parent = -1;        // index in the arena, -1 = virtual root
    double T = 0;           // virtual-root time
    std::vector<double> x;  // q_new (dof) then t_new
};

// Directed space-time distance (Eq. space-time-metric).
double rho_sigma(const double* q, double t, const double* qr, double tr, int sigma, int d, double v) {
    double Delta = (double)sigma * (tr - t);
    double D = dist(q, qr, d);
    if (!(Delta > 0.0) || !(D <= v * Delta)) return kInf;
    return std::sqrt((D * D + v * v * (tr - t) * (tr - t)) / 2.0);
}

// rho of an NN choice: the metric's value, or, for a vertex that a
// reduced-precision run found admissible while this FP64 run puts it just
// outside the speed cone (a flagged decision adopted in follow mode), the
// same formula without the cut, as that run steers with it.
double rho_sigma_adopted(const double* q, double t, const double* qr, double tr, int sigma, int d, double v) {
    const double r = rho_sigma(q, t, qr, tr, sigma, d, v);
    if (r < kInf) return r;
    const double D = dist(q, qr, d);
    return std::sqrt((D * D + v * v * (tr - t) * (tr - t)) / 2.0);
}

void note(double& slot, double v) {
    v = std::fabs(v);
    if (v < slot) slot = v;
}

// NN under rho_sigma over arena[0, n) restricted to nodes with troot < U when
// filter is set. Returns -1 if every rho is infinite. Tie: lowest index.
// Margins: the gap between the two smallest finite rho, and admissibility
// boundaries of nodes that would be competitive.
int nn_spacetime(const std::vector<Node>& A, int n, bool filter, double U, const double* qr, double tr,
                 int sigma, int d, double v, double* best_rho, Margin& M, double tol) {
    int best = -1;
    double b1 = kInf, b2 = kInf;
    for (int i = 0; i < n; ++i) {
        if (filter && !(A[i].troot < U)) continue;
        double r = rho_sigma(A[i].q.data(), A[i].t, qr, tr, sigma, d, v);
        if (r < b1) {
            b2 = b1;
            b1 = r;
            best = i;
        } else if (r < b2) {
            b2 = r;
        }
    }
    if (best >= 0 && b2 < kInf) note(M.nn, b2 - b1);
    for (int i = 0; i < n; ++i) {
        if (filter && !(A[i].troot < U)) continue;
        double Delta = (double)sigma * (tr - A[i].t);
        double D = dist(A[i].q.data(), qr, d);
        double madm = std::min(std::fabs(Delta), std::fabs(v * Delta - D));
        if (madm < tol) {
            double r = std::sqrt((D * D + v * v * (tr - A[i].t) * (tr - A[i].t)) / 2.0);
            if (r <= b1 + tol) note(M.nn, madm);
        }
    }
    *best_rho = b1;
    return best;
}

// Configuration-distance NN (root recycling) over arena[0, n). Tie: lowest index.
int nn_config(const std::vector<Node>& A, int n, const double* qr, int d, double* best_D, Margin& M) {
    int best = -1;
    double b1 = kInf, b2 = kInf;
    for (int i = 0; i < n; ++i) {
        double D = dist(A[i].q.data(), qr, d);
        if (D < b1) {
            b2 = b1;
            b1 = D;
            best = i;
        } else if (D < b2) {
            b2 = D;
        }
    }
    if (b2 < kInf) note(M.nn, b2 - b1);
    *best_D = b1;
    return best;
}

// Bridge rank (Algorithm 1, "Connect"; Sec. "Interval Root": a connection is
// ranked by arrival time, then by space-time distance). For an inserted node a
// the candidates are the vertices of the opposite start-of-iteration set that
// a can reach with an admissible edge (rho_sigma finite): a forward node looks
// at later vertices of the active backward trees (root time < U0), a backward
// node at earlier vertices of the forward tree. Key (arrival time = root time
// of the backward end, rho); ties go to the lowest (segment, index). Only the
// top-ranked candidate is ever validated (by the caller).
// margin: the smallest gap between the winner's key and a competing key, or
// between a competitive vertex and an admissibility boundary.
struct BridgeCand {
    int s = -1, i = -1;  // s: backward group / slot of the candidate, -1 for the forward tree
    double U = kInf, rho = kInf;
    double margin = kInf;
};

BridgeCand bridge_rank(const Node& a, bool forward, const std::vector<std::vector<Node>>& seg,
                       const std::vector<int>& seg_n, const std::vector<Node>& fwd, int fwd_n, double U0, int d,
                       double v, double tol) {
    BridgeCand c;
    double s1U = kInf, s1R = kInf;  // runner-up key
    auto consider = [&](int s, int i, double Uv, double r) {
        const bool better = (Uv < c.U) || (Uv == c.U && r < c.rho);
        if (better) {
            s1U = c.U;
            s1R = c.rho;
            c.U = Uv;
            c.rho = r;
            c.s = s;
            c.i = i;
        } else if ((Uv < s1U) || (Uv == s1U && r < s1R)) {
            s1U = Uv;
            s1R = r;
        }
    };
    // First pass: the ranking. Second pass: admissibility margins of vertices
    // whose key would be competitive with the winner.
    for (int pass = 0; pass < 2; ++pass) {
        if (forward) {
            for (int s = 0; s < (int)seg_n.size(); ++s) {
                for (int i = 0; i < seg_n[s]; ++i) {
                    const Node& b = seg[s][i];
                    if (!(b.troot < U0)) continue;
                    if (pass == 0) {
                        const double r = rho_sigma(a.q.data(), a.t, b.q.data(), b.t, 1, d, v);
                        if (r < kInf) consider(s, i, b.troot, r);
                        continue;
                    }
                    const double Delta = b.t - a.t, D = dist(a.q.data(), b.q.data(), d);
                    const double madm = std::min(std::fabs(Delta), std::fabs(v * Delta - D));
                    const double ru = std::sqrt((D * D + v * v * Delta * Delta) / 2.0);
                    if (madm < tol && b.troot <= c.U + tol && ru <= c.rho + tol) note(c.margin, madm);
                }
            }
        } else {
            for (int i = 0; i < fwd_n; ++i) {
                const Node& b = fwd[i];
                if (pass == 0) {
                    const double r = rho_sigma(b.q.data(), b.t, a.q.data(), a.t, 1, d, v);
                    if (r < kInf) consider(-1, i, a.troot, r);
                    continue;
                }
                const double Delta = a.t - b.t, D = dist(a.q.data(), b.q.data(), d);
                const double madm = std::min(std::fabs(Delta), std::fabs(v * Delta - D));
                const double ru = std::sqrt((D * D + v * v * Delta * Delta) / 2.0);
                if (madm < tol && ru <= c.rho + tol) note(c.margin, madm);
            }
        }
    }
    if (c.i >= 0) {
        if (s1U == c.U && s1R < kInf) note(c.margin, s1R - c.rho);
        if (s1U != c.U && s1U < kInf) note(c.margin, s1U - c.U);
    }
    return c;
}

// Publish order (Sec. "GPU-Parallel Space-Time Forest": workers publish
// improved solutions atomically; batch-synchronous reading: of an iteration's
// successful bridges the lexicographically smallest (U, C, worker) wins).
bool publish_before(double U1, double C1, int w1, double U2, double C2, int w2) {
    if (U1 != U2) return U1 < U2;
    if (C1 != C2) return C1 < C2;
    return w1 < w2;
}

// Follow mode (parity of a reduced-precision device run against this FP64
// run). At a decision whose FP64 margin lies below the flag threshold the
// oracle adopts the device's recorded choice and continues; at any other
// decision a differing device choice is an unflagged mismatch: it is recorded
// (the parity tests require none) and adopted, so that the comparison still
// covers the rest of the run.
struct Follow {
    const int* rec = nullptr;
    int iters = 0, W = 0;
    const int* at(int k, int w) const {
        if (!rec || k >= iters) return nullptr;
        return rec + ((size_t)k * W + w) * kTraceInts;
    }
};

class Planner {
public:
    Planner(const Problem& P, const Params& prm) : P(P), prm(prm) {}

    Result run();

private:
    const Problem& P;
    const Params& prm;
    Result R;
    GoalGrid grid;
    IntervalAlloc alloc;
    Learned learned;
    Follow F;
    long kend = 0;  // first grid index with k dt >= H (recycling roots lie in [L_grid, H))

    int d() const { return P.dof; }
    // One decision: `mine` with FP64 margin flagged or not, against the device
    // record's value `dev` when following (dev_rec != nullptr).
    int decide(int k, int w, int kind, int mine, const void* dev_rec, int dev, bool flagged) {
        if (!dev_rec) return mine;
        if (flagged) {
            R.followed[kind]++;
            if (dev != mine) R.flagged_diff[kind]++;
            return dev;
        }
        if (dev != mine) {
            R.unflagged.push_back(k);
            R.unflagged.push_back(w);
            R.unflagged.push_back(kind);
            return dev;
        }
        return mine;
    }
    bool decide_flag(int k, int w, int kind, bool mine, const int* dev_rec, int bit, bool flagged) {
        const int dev = dev_rec ? ((dev_rec[0] & bit) ? 1 : 0) : 0;
        return decide(k, w, kind, mine ? 1 : 0, dev_rec, dev, flagged) != 0;
    }
    // Edge check with follow decisions on its count and verdict.
    bool check_edge_follow(int k, int w, const double* qa, double ta, const double* qb, double tb, Margin& M,
                           const int* dv, int count_field, int kind_count, int hit_bit, int kind_hit, int* count_out) {
        double clr, im = kInf, bm = kInf;
        int c = 0;
        bool ok;
        if (prm.continuous) {
            // The count only marks the entry (the verdict is closed-form).
            ok = edge_free_continuous(P, qa, ta, qb, tb, &clr);
            c = edge_check_count(P, qa, ta, qb, tb, prm.res, nullptr);
        } else {
            c = edge_check_count(P, qa, ta, qb, tb, prm.res, &im);
            c = decide(k, w, kind_count, c, dv, dv ? dv[count_field] : 0, im < prm.flag_tol);
            ok = edge_free(P, qa, ta, qb, tb, prm.res, &clr, nullptr, nullptr, &bm, c);
            note(M.count, im);
            note(M.bounds, bm);
        }
        note(M.clearance, clr);
        const bool flagged = std::fabs(clr) < prm.flag_clear || std::fabs(bm) < prm.flag_tol;
        const bool hit = decide_flag(k, w, kind_hit, !ok, dv, hit_bit, flagged);
        *count_out = c;
        return !hit;
    }
    void init_recycling();
    void recycle(double U);
    Proposal propose_interval(int k, int w, const std::vector<int>& seg_n, int fwd_n, double U0,
                              const std::vector<int>& group_active, Margin& M, int* rec, double* rd);
    Proposal propose_recycling(int k, int w, const std::vector<int>& seg_n, int fwd_n,
                               const std::vector<int>& active_slots, Margin& M, int* rec);
    void extract_path();
};

void Planner::init_recycling() {
    // Reading (root initialisation): the grid indices of [L_grid, H) are split
    // into N equal integer ranges; slot i takes the first collision-free goal
    // check of its range, scanning upward; none found leaves the slot empty.
    long K = kend - grid.kmin;
    R.slots.assign(prm.N, Slot());
    R.seg.assign(prm.N, {});
    for (int i = 0; i < prm.N; ++i) {
        long a = grid.kmin + (K * i) / prm.N;
        long b = grid.kmin + (K * (i + 1)) / prm.N;
        for (long k = a; k < b; ++k) {
            if (grid.is_free(k)) {
                Slot& s = R.slots[i];
                s.has_root = true;
                s.active = true;
                s.k = k;
                s.T = (double)k * prm.dt;
                s.gen = 0;
                Node root;
                root.q = P.qg;
                root.t = s.T;
                root.parent = -1;
                root.troot = s.T;
                root.cost = 0.0;
                root.tree = 0;
                root.iter = -1;
                R.seg[i].push_back(root);
                break;
            }
        }
    }
}

void Planner::recycle(double U) {
    std::vector<int> rep = recycle_rule(R.slots, U, grid.kmin, prm.dt, [&](long k) { return grid.is_free(k); });
    for (int i : rep) {
        // The slot's old tree is retired; a fresh root (q_g, T_i') with no
        // children takes its place.
        const Slot& s = R.slots[i];
        Node root;
        root.q = P.qg;
        root.t = s.T;
        root.parent = -1;
        root.troot = s.T;
        root.cost = 0.0;
        root.tree = s.gen;
        root.iter = R.iters - 1;
        R.seg[i].assign(1, root);
    }
}

Proposal Planner::propose_interval(int k, int w, const std::vector<int>& seg_n, int fwd_n, double U0,
                                   const std::vector<int>& group_active, Margin& M, int* rec, double* rd) {
    Proposal pr;
    int dd = d();
    const int* dv = F.at(k, w);
    Draws dr;
    dr.fill(prm.seed, prm.problem_id, (uint32_t)k, (uint32_t)w, learned.on ? 17 : 5 + dd);
    const bool lrn = learned.on && (dr.raw[12] >> 8) < kThrLearned;
    pr.forward = ((w + k) % 2) == 0;
    pr.forward = decide_flag(k, w, kKDirection, pr.forward, dv, kTrFwd, false);
    int g = dr.group(0, prm.N);
    g = decide(k, w, kKGroup, g, dv, dv ? dv[1] : 0, false);
    pr.seg = g;
    rec[0] |= (pr.forward ? kTrFwd : 0) | (lrn ? kTrLearned : 0);
    rec[1] = g;
    bool guided;
    double walk;
    double T = sample_goal_time(alloc, g, dr.u(1), dr.u(2), prm.p_guided, &guided, &walk);
    // The guided measure below U-bar changes discontinuously where a guided
    // window starts or ends at U-bar, and the piece walk jumps gaps: margins
    // of the goal-time draw (a reduced-precision U moves U-bar slightly).
    double tmargin = walk;
    if (dr.u(1) < prm.p_guided) {
        tmargin = std::min(tmargin, alloc.group_measure[g]);
        for (const auto& wdw : alloc.windows)
            tmargin = std::min(tmargin, std::min(std::fabs(wdw.first - alloc.Ubar), std::fabs(wdw.second - alloc.Ubar)));
    }
    const bool tflag = tmargin < prm.flag_tol;
    guided = decide_flag(k, w, kKGuided, guided, dv, kTrGuided, tflag);
    if (guided) rec[0] |= kTrGuided;
    if (lrn) {
        double cm;
        double Tl = learned_T(learned, dr, &cm);
        int comp = 0;
        while (comp < 7 && !(dr.u(14) < learned.cw[comp])) ++comp;
        const int comp_f = decide(k, w, kKLearnedComp, comp, dv, dv ? dv[8] : 0, cm < prm.flag_tol);
        if (comp_f != comp) {
            // Adopted component: the same normal draw around its mean.
            const double u1 = 1.0 - dr.u(15), u2 = dr.u(16);
            const double z = std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586476925 * u2);
            Tl = learned.mu[comp_f] + learned.sig[comp_f] * z;
        }
        rec[8] = comp_f;
        const double glo = alloc.Lg + (double)g * alloc.width;
        note(M.interval, cm);
        note(M.bounds, Tl - glo);
        note(M.bounds, glo + alloc.width - Tl);
        const double mb = std::min(std::fabs(Tl - glo), std::fabs(glo + alloc.width - Tl));
        const bool take = decide_flag(k, w, kKLearnedT, Tl >= glo && Tl < glo + alloc.width, dv, kTrLearnedT,
                                      mb < prm.flag_tol);
        if (take) {
            T = Tl;
            rec[0] |= kTrLearnedT;
        }
    }
    if (dv) {
        // The goal time itself (as stored by the device, float): beyond the
        // rounding of a float time it must agree unless its draw was flagged.
        float tf;
        std::memcpy(&tf, &dv[9], sizeof(tf));
        const double Td = (double)tf;
        if (std::fabs(Td - T) > 4e-7 * std::max(1.0, std::fabs(T)) + prm.flag_tol * 1e-2) {
            if (tflag) {
                R.followed[kKGoalTime]++;
                R.flagged_diff[kKGoalTime]++;
            } else {
                R.unflagged.push_back(k);
                R.unflagged.push_back(w);
                R.unflagged.push_back(kKGoalTime);
            }
            T = Td;
        }
    }
    pr.T = T;
    rd[0] = T;
    {
        const float tf = (float)T;
        std::memcpy(&rec[9], &tf, sizeof(tf));
    }
    // A new root is checked for collision at the goal time drawn for it; if
    // it collides, the worker makes no attempt this iteration (Algorithm 2).
    {
        double cl;
        const bool free = state_free(P, P.qg.data(), T, &cl);
        R.root_checked++;
        note(M.clearance, cl);
        // The device checks the root together with the extension edge, so its
        // verdict exists only for workers that emitted one.
        const int* dvr = (dv && (dv[0] & kTrEmit)) ? dv : nullptr;
        const bool hit = decide_flag(k, w, kKRoot, !free, dvr, kTrRootHit, std::fabs(cl) < prm.flag_clear);
        if (hit) {
            rec[0] |= kTrRootHit;
            return pr;
        }
    }
    // Conditional query sample (Eq. conditional-query-time).
    std::vector<double> qr(dd);
    for (int j = 0; j < dd; ++j) qr[j] = P.qlo[j] + dr.u(4 + j) * (P.qhi[j] - P.qlo[j]);
    if (lrn) learned_q(learned, dr, P.qlo, P.qhi, dd, qr.data());
    double lo = dist(P.qs.data(), qr.data(), dd) / P.vmax;
    double hi = T - dist(qr.data(), P.qg.data(), dd) / P.vmax;
    rd[2] = lo;
    rd[3] = hi;
    note(M.interval, hi - lo);
    const bool sampled = decide_flag(k, w, kKWindow, !(lo > hi), dv, kTrSampled, std::fabs(hi - lo) < prm.flag_tol);
    if (!sampled) return pr;
    rec[0] |= kTrSampled;
    double tr = lo + dr.u(4 + dd) * (hi - lo);
    rd[1] = tr;

    // Source set and NN (Algorithm 1).
    const double* qn;
    double tn;
    double rho;
    if (pr.forward) {
        Margin Mw;
        int i = nn_spacetime(R.fwd, fwd_n, false, U0, qr.data(), tr, 1, dd, P.vmax, &rho, Mw, prm.flag_tol);
        note(M.nn, Mw.nn);
        i = decide(k, w, kKParent, i, dv, dv ? dv[2] : 0, Mw.nn < prm.flag_tol);
        rec[2] = i;
        if (i < 0) return pr;
        if (i >= fwd_n) return pr;  // an adopted index outside the set (already counted as a mismatch)
        rho = rho_sigma_adopted(R.fwd[i].q.data(), R.fwd[i].t, qr.data(), tr, 1, dd, P.vmax);
        pr.parent = i;
        qn = R.fwd[i].q.data();
        tn = R.fwd[i].t;
    } else {
        bool use_new = (group_active[g] == 0) || (dr.u(3) <= prm.p_new);
        use_new = decide_flag(k, w, kKVirtual, use_new, dv, kTrVirtual, false);
        if (use_new) {
            rec[0] |= kTrVirtual;
            rho = rho_sigma(P.qg.data(), T, qr.data(), tr, -1, dd, P.vmax);
            // Admissibility of the virtual root (rho finite) is an emit decision.
            const double Delta = T - tr, D = dist(P.qg.data(), qr.data(), dd);
            const double madm = std::min(std::fabs(Delta), std::fabs(P.vmax * Delta - D));
            note(M.bounds, madm);
            if (!(rho < kInf)) {
                const bool emit = decide_flag(k, w, kKEmit, false, dv, kTrEmit, madm < prm.flag_tol);
                if (!emit) return pr;
                rho = std::sqrt((D * D + P.vmax * P.vmax * Delta * Delta) / 2.0);
            }
            pr.parent = -1;
            rec[2] = -1;
            qn = P.qg.data();
            tn = T;
        } else {
            Margin Mw;
            int i = nn_spacetime(R.seg[g], seg_n[g], true, U0, qr.data(), tr, -1, dd, P.vmax, &rho, Mw,
                                 prm.flag_tol);
            note(M.nn, Mw.nn);
            i = decide(k, w, kKParent, i, dv, dv ? dv[2] : 0, Mw.nn < prm.flag_tol);
            rec[2] = i;
            if (i < 0 || i >= seg_n[g]) return pr;
            rho = rho_sigma_adopted(R.seg[g][i].q.data(), R.seg[g][i].t, qr.data(), tr, -1, dd, P.vmax);
            pr.parent = i;
            qn = R.seg[g][i].q.data();
            tn = R.seg[g][i].t;
        }
    }
    // Steering: x_new = x_n + alpha (x_r - x_n), alpha = min(1, eta / rho).
    double alpha = std::min(1.0, prm.eta / rho);
    pr.x.assign(dd + 1, 0.0);
    for (int j = 0; j < dd; ++j) pr.x[j] = qn[j] + alpha * (qr[j] - qn[j]);
    double tnew = tn + alpha * (tr - tn);
    pr.x[dd] = tnew;
    note(M.bounds, tnew);
    note(M.bounds, prm.H - tnew);
    const double mh = std::min(std::fabs(tnew), std::fabs(prm.H - tnew));
    const bool emit = decide_flag(k, w, kKEmit, !(tnew < 0.0 || tnew > prm.H), dv, kTrEmit, mh < prm.flag_tol);
    if (!emit) return pr;
    rec[0] |= kTrEmit;
    int c;
    const bool ok = check_edge_follow(k, w, qn, tn, pr.x.data(), tnew, M, dv, 3, kKExtCount, kTrExtHit, kKExtHit, &c);
    rec[3] = c;
    if (!ok) rec[0] |= kTrExtHit;
    R.ext_checked++;
    pr.ok = ok;
    return pr;
}

Proposal Planner::propose_recycling(int k, int w, const std::vector<int>& seg_n, int fwd_n,
                                    const std::vector<int>& active_slots, Margin& M, int* rec) {
    Proposal pr;
    int dd = d();
    const int* dv = F.at(k, w);
    pr.forward = ((w + k) % 2) == 0;
    pr.forward = decide_flag(k, w, kKDirection, pr.forward, dv, kTrFwd, false);
    rec[0] |= pr.forward ? kTrFwd : 0;
    // Reading (round-robin): the backward worker with ordinal floor(w/2) in this
    // iteration takes active slot number ordinal mod (#active), in slot order.
    if (!pr.forward) {
        const int slot = active_slots.empty() ? -1 : active_slots[(w / 2) % active_slots.size()];
        pr.seg = decide(k, w, kKGroup, slot, dv, dv ? dv[1] : 0, false);
        rec[1] = pr.seg;
        if (pr.seg < 0 || pr.seg >= prm.N) return pr;
    }
    rec[0] |= kTrSampled;
    Draws dr;
    dr.fill(prm.seed, prm.problem_id, (uint32_t)k, (uint32_t)w, learned.on ? 17 : 4 + dd);
    std::vector<double> qr(dd);
    for (int j = 0; j < dd; ++j) qr[j] = P.qlo[j] + dr.u(4 + j) * (P.qhi[j] - P.qlo[j]);
    if (learned.on && (dr.raw[12] >> 8) < kThrLearned) {
        rec[0] |= kTrLearned;
        learned_q(learned, dr, P.qlo, P.qhi, dd, qr.data());
    }
    const std::vector<Node>& A = pr.forward ? R.fwd : R.seg[pr.seg];
    int n = pr.forward ? fwd_n : seg_n[pr.seg];
    double D;
    Margin Mw;
    int i = nn_config(A, n, qr.data(), dd, &D, Mw);
    note(M.nn, Mw.nn);
    i = decide(k, w, kKParent, i, dv, dv ? dv[2] : 0, Mw.nn < prm.flag_tol);
    rec[2] = i;
    if (i < 0 || i >= n) return pr;
    D = dist(A[i].q.data(), qr.data(), dd);
    note(M.bounds, D);
    pr.parent = i;
    const double* qn = A[i].q.data();
    double tn = A[i].t;
    // Max-speed extension (Eq. max-speed-extension), configuration step capped at eta.
    double s = D > 0.0 ? std::min(1.0, prm.eta / D) : 0.0;
    pr.x.assign(dd + 1, 0.0);
    for (int j = 0; j < dd; ++j) pr.x[j] = qn[j] + s * (qr[j] - qn[j]);
    double Dn = dist(qn, pr.x.data(), dd);
    double tnew = tn + (pr.forward ? 1.0 : -1.0) * Dn / P.vmax;
    pr.x[dd] = tnew;
    note(M.bounds, tnew);
    note(M.bounds, prm.H - tnew);
    const double mh = std::min(std::min(std::fabs(tnew), std::fabs(prm.H - tnew)), D);
    const bool emit = decide_flag(k, w, kKEmit, D > 0.0 && !(tnew < 0.0 || tnew > prm.H), dv, kTrEmit,
                                  mh < prm.flag_tol);
    if (!emit) return pr;
    rec[0] |= kTrEmit;
    int c;
    const bool ok = check_edge_follow(k, w, qn, tn, pr.x.data(), tnew, M, dv, 3, kKExtCount, kTrExtHit, kKExtHit, &c);
    rec[3] = c;
    if (!ok) rec[0] |= kTrExtHit;
    R.ext_checked++;
    pr.ok = ok;
    return pr;
}

void Planner::extract_path() {
    R.path.clear();
    if (R.inc_fwd < 0) return;
    int dd = d();
    std::vector<int> chain;
    for (int i = R.inc_fwd; i >= 0; i = R.fwd[i].parent) chain.push_back(i);
    std::reverse(chain.begin(), chain.end());
    for (int i : chain) {
        for (int j = 0; j < dd; ++j) R.path.push_back(R.fwd[i].q[j]);
        R.path.push_back(R.fwd[i].t);
    }
    const std::vector<Node>& B = R.seg[R.inc_seg];
    for (int i = R.inc_bwd; i >= 0; i = B[i].parent) {
        for (int j = 0; j < dd; ++j) R.path.push_back(B[i].q[j]);
        R.path.push_back(B[i].t);
    }
}

Result Planner::run() {
    int dd = d();
    if (prm.proposal) build_learned(learned, prm.proposal, P.qlo, P.qhi, P.qs, P.qg, dd, prm.H);
    F.rec = prm.follow_rec;
    F.iters = prm.follow_rec ? prm.follow_iters : 0;
    F.W = prm.W;
    R.dof = dd;
    R.N = prm.N;
    R.variant = prm.variant;
    // Forward tree rooted at (q_s, 0).
    Node s0;
    s0.q = P.qs;
    s0.t = 0.0;
    s0.parent = -1;
    s0.troot = 0.0;
    s0.cost = 0.0;
    s0.tree = 0;
    s0.iter = -1;
    R.fwd.push_back(s0);

    // Early return when q_s = q_g and x_s is free (first line of Algorithms 2, 3).
    bool same = true;
    for (int j = 0; j < dd; ++j)
        if (P.qs[j] != P.qg[j]) same = false;
    if (same && state_free(P, P.qs.data(), 0.0, nullptr)) {
        R.U = 0.0;
        R.C = 0.0;
        R.inc_fwd = 0;
        R.path.assign(P.qs.begin(), P.qs.end());
        R.path.push_back(0.0);
        R.seg.assign(prm.N, {});
        R.status = 0;
        return R;
    }
    if (!state_free(P, P.qs.data(), 0.0, nullptr)) {
        R.seg.assign(prm.N, {});
        R.status = 5;
        return R;
    }

    build_goal_grid(P, prm.H, prm.dt, grid);
    if (prm.follow_grid) {
        // Goal checks: adopt the device's verdict inside the clearance band.
        for (size_t i = 0; i < grid.free.size(); ++i) {
            const int dev = (int)i < prm.follow_nk ? (prm.follow_grid[i] ? 1 : 0) : 0;
            const bool flagged = std::fabs(grid.clearance[i]) < prm.flag_clear;
            grid.free[i] = (char)decide(-1, (int)i, kKGrid, grid.free[i] ? 1 : 0, prm.follow_grid, dev, flagged);
        }
    }
    R.goal_clearance = grid.clearance;
    R.goal_kmin = grid.kmin;
    kend = grid.kmin;
    while ((double)kend * prm.dt < prm.H) ++kend;

    if (prm.variant == 0) {
        alloc.Lg = grid.Lg;
        alloc.H = prm.H;
        alloc.dt = prm.dt;
        alloc.N = prm.N;
        if (grid.kmax >= grid.kmin) build_windows(alloc, grid.kmin, grid.kmax, grid.free.data());
        partition(alloc, kInf);
        R.seg.assign(prm.N, {});
    } else {
        init_recycling();
    }

    const double nan = std::nan("");
    for (int k = 0; k < prm.max_iters; ++k) {
        if (prm.variant == 0 && !(grid.Lg < std::min(prm.H, R.U))) break;
        Margin M;
        const double U0 = R.U, C0 = R.C;
        const int fwd_n = (int)R.fwd.size();
        std::vector<int> seg_n(prm.N);
        for (int i = 0; i < prm.N; ++i) seg_n[i] = (int)R.seg[i].size();
        std::vector<int> group_active(prm.N, 0);
        std::vector<int> active_slots;
        if (prm.variant == 0) {
            for (const Tree& t : R.trees)
                if (t.T < U0) group_active[t.group]++;
        } else {
            for (int i = 0; i < prm.N; ++i)
                if (R.slots[i].active) active_slots.push_back(i);
        }
        const size_t rec0 = R.trace.size();
        R.trace.resize(rec0 + (size_t)prm.W * kTraceInts, 0);
        R.trace_d.resize(R.trace_d.size() + (size_t)prm.W * 4, nan);
        int* recs = &R.trace[rec0];
        double* rds = &R.trace_d[R.trace_d.size() - (size_t)prm.W * 4];
        for (int w = 0; w < prm.W; ++w) {
            int* r = recs + (size_t)w * kTraceInts;
            r[1] = r[2] = r[4] = r[5] = r[7] = r[8] = -1;
        }

        // 1. Every worker proposes against the start-of-iteration state.
        std::vector<Proposal> props(prm.W);
        for (int w = 0; w < prm.W; ++w) {
            int* r = recs + (size_t)w * kTraceInts;
            props[w] = (prm.variant == 0)
                           ? propose_interval(k, w, seg_n, fwd_n, U0, group_active, M, r, rds + (size_t)w * 4)
                           : propose_recycling(k, w, seg_n, fwd_n, active_slots, M, r);
        }

        // 2. Ordered insertion (worker order).
        struct Inserted {
            int w;
            bool forward;
            int seg;
            int idx;
        };
        std::vector<Inserted> ins;
        for (int w = 0; w < prm.W; ++w) {
            Proposal& pr = props[w];
            if (!pr.ok) continue;
            Node nd;
            nd.q.assign(pr.x.begin(), pr.x.begin() + dd);
            nd.t = pr.x[dd];
            nd.iter = k;
            int* r = recs + (size_t)w * kTraceInts;
            r[0] |= kTrInserted;
            if (pr.forward) {
                const Node& par = R.fwd[pr.parent];
                nd.parent = pr.parent;
                nd.troot = 0.0;
                nd.cost = par.cost + dist(par.q.data(), nd.q.data(), dd);
                nd.tree = 0;
                R.fwd.push_back(nd);
                ins.push_back({w, true, -1, (int)R.fwd.size() - 1});
            } else {
                std::vector<Node>& A = R.seg[pr.seg];
                if (pr.parent < 0) {
                    // Materialise the virtual root as a new backward tree.
                    Node root;
                    root.q = P.qg;
                    root.t = pr.T;
                    root.parent = -1;
                    root.troot = pr.T;
                    root.cost = 0.0;
                    root.tree = (int)R.trees.size();
                    root.iter = k;
                    R.trees.push_back({pr.seg, pr.T});
                    A.push_back(root);
                    nd.parent = (int)A.size() - 1;
                } else {
                    nd.parent = pr.parent;
                }
                const Node& par = A[nd.parent];
                nd.troot = par.troot;
                nd.cost = par.cost + dist(par.q.data(), nd.q.data(), dd);
                nd.tree = par.tree;
                A.push_back(nd);
                ins.push_back({w, false, pr.seg, (int)A.size() - 1});
            }
            r[7] = ins.back().idx;
            R.inserted++;
        }

        // 3. Bridge: the best-ranked admissible vertex of the opposite
        // start-of-iteration set is validated if it would improve (U0, C0).
        // 4. Publish: lexicographic min of (U, C, worker).
        int best_w = -1;
        double bestU = kInf, bestC = kInf;
        int best_f = -1, best_s = -1, best_b = -1;
        struct Success {
            int w;
            double U, C;
            int f, s, b;
        };
        std::vector<Success> wins;
        const double ctol = prm.flag_tol * std::max(1.0, std::fabs(C0) < kInf ? std::fabs(C0) : 1.0);
        for (const Inserted& in : ins) {
            int* r = recs + (size_t)in.w * kTraceInts;
            const int* dv = F.at(k, in.w);
            const Node& a = in.forward ? R.fwd[in.idx] : R.seg[in.seg][in.idx];
            BridgeCand bc = bridge_rank(a, in.forward, R.seg, seg_n, R.fwd, fwd_n, U0, dd, P.vmax, prm.flag_tol);
            note(M.rank, bc.margin);
            const bool rflag = bc.margin < prm.flag_tol;
            const bool has = decide_flag(k, in.w, kKBrCand, bc.i >= 0, dv, kTrBrCand, rflag);
            if (!has) continue;
            int cs = decide(k, in.w, kKBrCand, bc.s, dv, dv ? dv[4] : 0, rflag);
            int ci = decide(k, in.w, kKBrCand, bc.i, dv, dv ? dv[5] : 0, rflag);
            if (in.forward ? (cs < 0 || cs >= prm.N || ci < 0 || ci >= seg_n[cs]) : (ci < 0 || ci >= fwd_n))
                continue;  // an adopted candidate outside the set (already counted as a mismatch)
            r[0] |= kTrBrCand;
            r[4] = in.forward ? cs : -1;
            r[5] = ci;
            const Node& b = in.forward ? R.seg[cs][ci] : R.fwd[ci];
            const Node& fnode = in.forward ? a : b;
            const Node& bnode = in.forward ? b : a;
            double Dab = dist(fnode.q.data(), bnode.q.data(), dd);
            double Uc = bnode.troot;
            double Cc = fnode.cost + Dab + bnode.cost;
            bool improves = (Uc < U0) || (Uc == U0 && Cc < C0);
            if (Uc != U0 && U0 < kInf) note(M.rank, Uc - U0);
            if (Uc == U0) note(M.cost, Cc - C0);
            const bool iflag = (Uc != U0 && U0 < kInf && std::fabs(Uc - U0) < prm.flag_tol) ||
                               (Uc == U0 && std::fabs(Cc - C0) < ctol);
            improves = decide_flag(k, in.w, kKBrEmit, improves, dv, kTrBrEmit, iflag);
            if (!improves) continue;
            r[0] |= kTrBrEmit;
            int c;
            const bool ok = check_edge_follow(k, in.w, fnode.q.data(), fnode.t, bnode.q.data(), bnode.t, M, dv, 6,
                                              kKBrCount, kTrBrHit, kKBrHit, &c);
            r[6] = c;
            R.bridge_checked++;
            if (!ok) {
                r[0] |= kTrBrHit;
                continue;
            }
            wins.push_back({in.w, Uc, Cc, in.forward ? in.idx : ci, in.forward ? cs : in.seg,
                            in.forward ? ci : in.idx});
        }
        // Publish: lexicographic (U, C, worker) minimum of the successes.
        int wi = -1;
        for (int i = 0; i < (int)wins.size(); ++i)
            if (wi < 0 || publish_before(wins[i].U, wins[i].C, wins[i].w, wins[wi].U, wins[wi].C, wins[wi].w)) wi = i;
        bool pflag = false;
        if (wi >= 0) {
            const double ptol = prm.flag_tol * std::max(1.0, std::fabs(wins[wi].C));
            for (int i = 0; i < (int)wins.size(); ++i) {
                if (i == wi) continue;
                if (wins[i].U != wins[wi].U) {
                    note(M.rank, wins[i].U - wins[wi].U);
                    pflag = pflag || std::fabs(wins[i].U - wins[wi].U) < prm.flag_tol;
                } else {
                    note(M.cost, wins[i].C - wins[wi].C);
                    pflag = pflag || std::fabs(wins[i].C - wins[wi].C) < ptol;
                }
            }
        }
        if (F.rec && k < F.iters) {
            int dev_w = -1;
            for (int w = 0; w < prm.W; ++w)
                if (F.at(k, w)[0] & kTrWinner) dev_w = w;
            const int mine_w = wi >= 0 ? wins[wi].w : -1;
            const int chosen = decide(k, mine_w >= 0 ? mine_w : dev_w, kKWinner, mine_w, F.rec, dev_w, pflag);
            wi = -1;
            for (int i = 0; i < (int)wins.size(); ++i)
                if (wins[i].w == chosen) wi = i;
        }
        if (wi >= 0) {
            const Success& s = wins[wi];
            recs[(size_t)s.w * kTraceInts] |= kTrWinner;
            best_w = s.w;
            bestU = s.U;
            bestC = s.C;
            best_f = s.f;
            best_s = s.s;
            best_b = s.b;
        }
        R.iters = k + 1;
        bool decreased = false;
        if (best_w >= 0) {
            decreased = bestU < R.U;
            R.U = bestU;
            R.C = bestC;
            R.inc_fwd = best_f;
            R.inc_seg = best_s;
            R.inc_bwd = best_b;
            if (R.first_iter < 0) R.first_iter = k;
        }
        // 5. Allocation update when U decreased.
        if (decreased) {
            if (prm.variant == 0) {
                partition(alloc, R.U);
            } else if (prm.variant == 1) {
                recycle(R.U);
            } else {
                // No recycling (Sec. Goal-Time Range and Capacity Ablations):
                // the fixed forest keeps its roots; those at T >= U go inactive.
                for (Slot& sl : R.slots)
                    if (sl.has_root && sl.T >= R.U) sl.active = false;
            }
        }
        R.U_hist.push_back(R.U);
        R.C_hist.push_back(R.C);
        R.margin_hist.push_back(M.min_all());
        double mt[6] = {M.nn, M.count, M.interval, M.bounds, M.rank, M.clearance};
        R.margin_types.insert(R.margin_types.end(), mt, mt + 6);
        R.clear_hist.push_back(M.clearance);
    }
    extract_path();
    R.status = (R.inc_fwd >= 0) ? 0 : 5;
    return R;
}

// ---------------------------------------------------------------------------
// C interface (ctypes).
// ---------------------------------------------------------------------------
}  // namespace

extern "C" {

typedef struct {
    int dof;
    int arm;
    const double* dh;
    const double* qlo;
    const double* qhi;
    int n_sph;
    const double* sph;  // [S][5] link, x, y, z, r
    double vmax;
    int n_obs;
    int n_way;
    const double* obs_r;
    const double* way;  // [M][K][4]
    const double* qs;
    const double* qg;
    int self_collision;  // arms: also test sphere pairs of non-adjacent frames
} orc_problem;

typedef struct {
    int variant;
    int n_roots;
    int workers;
    int max_iters;
    double eta, res, dt, p_new, p_guided, H;
    unsigned long long seed;
    unsigned int problem_id;
    double flag_tol, flag_clear;
    int learned;              /* 1: learned branch with proposal[160] */
    const double* proposal;
    double t_offset;          /* absolute time of local time 0 */
    int continuous;           /* 1: closed-form edge validation (point robots) */
    const int* follow_rec;    /* follow mode: device decision records [iters][W][10], or NULL */
    int follow_iters;
    const unsigned char* follow_grid;  /* device goal-grid free flags, or NULL */
    int follow_nk;
} orc_params;

static Problem to_problem(const orc_problem* p) {
    Problem P;
    P.dof = p->dof;
    P.arm = p->arm != 0;
    if (P.arm) P.dh.assign(p->dh, p->dh + 4 * p->dof);
    P.qlo.assign(p->qlo, p->qlo + p->dof);
    P.qhi.assign(p->qhi, p->qhi + p->dof);
    for (int s = 0; s < p->n_sph; ++s) {
        P.sph_link.push_back((int)p->sph[5 * s]);
        for (int i = 0; i < 3; ++i) P.sph_p.push_back(p->sph[5 * s + 1 + i]);
        P.sph_r.push_back(p->sph[5 * s + 4]);
    }
    P.vmax = p->vmax;
    P.n_obs = p->n_obs;
    P.n_way = p->n_way;
    P.obs_r.assign(p->obs_r, p->obs_r + p->n_obs);
    P.way.assign(p->way, p->way + (size_t)p->n_obs * p->n_way * 4);
    P.qs.assign(p->qs, p->qs + p->dof);
    P.qg.assign(p->qg, p->qg + p->dof);
    if (p->self_collision && P.arm) {
        // Reading (self-collision, not in the paper's queries): spheres on the
        // same or adjacent frames never count; pairs already overlapping at the
        // zero configuration are treated as permanent contacts and ignored.
        std::vector<double> zero(P.dof, 0.0), c;
        std::vector<Frame> frames;
        forward_kinematics(P, zero.data(), frames);
        sphere_centres(P, frames, c);
        const int S = (int)P.sph_r.size();
        for (int a = 0; a < S; ++a)
            for (int b = a + 1; b < S; ++b) {
                if (std::abs(P.sph_link[a] - P.sph_link[b]) < 2) continue;
                double dx = c[3 * a] - c[3 * b], dy = c[3 * a + 1] - c[3 * b + 1], dz = c[3 * a + 2] - c[3 * b + 2];
                double rr = P.sph_r[a] + P.sph_r[b];
                if (dx * dx + dy * dy + dz * dz < rr * rr) continue;
                P.self_pairs.push_back({a, b});
            }
    }
    return P;
}

// Self-collision pairs of a problem (pins): [n][2].
int orc_self_pairs(const orc_problem* prob, int* pairs, int cap) {
    Problem P = to_problem(prob);
    int n = (int)P.self_pairs.size();
    for (int i = 0; i < n && i < cap; ++i) {
        pairs[2 * i] = P.self_pairs[i].first;
        pairs[2 * i + 1] = P.self_pairs[i].second;
    }
    return n;
}

void orc_philox4x32_10(const unsigned int ctr[4], const unsigned int key[2], unsigned int out[4]) {
    philox4x32_10(ctr, key, out);
}

// Sphere centres [S][3] and frame origins [dof+1][3], rotations [dof+1][9].
void orc_fk(const orc_problem* prob, const double* q, double* centres, double* origins, double* rots) {
    Problem P = to_problem(prob);
    std::vector<Frame> frames;
    std::vector<double> c;
    forward_kinematics(P, q, frames);
    sphere_centres(P, frames, c);
    if (centres) std::memcpy(centres, c.data(), c.size() * sizeof(double));
    for (size_t f = 0; f < frames.size(); ++f) {
        if (origins) std::memcpy(origins + 3 * f, frames[f].o, 3 * sizeof(double));
        if (rots) std::memcpy(rots + 9 * f, frames[f].R, 9 * sizeof(double));
    }
}

void orc_obstacle_position(const orc_problem* prob, int m, double t, double* out) {
    Problem P = to_problem(prob);
    obstacle_position(P, m, t, out);
}

int orc_state_free(const orc_problem* prob, const double* q, double t, double* clearance) {
    Problem P = to_problem(prob);
    return state_free(P, q, t, clearance) ? 1 : 0;
}

// Batch edge check: edges given in double, [n][dof] and [n].
void orc_check_edges(const orc_problem* prob, int n, const double* qa, const double* ta, const double* qb,
                     const double* tb, double res, unsigned char* verdict, double* clearance, int* nchk,
                     double* int_margin, double* bound_margin) {
    Problem P = to_problem(prob);
    int d = P.dof;
    for (int e = 0; e < n; ++e) {
        double clr, im, bm;
        int c;
        bool ok = edge_free(P, qa + (size_t)e * d, ta[e], qb + (size_t)e * d, tb[e], res, &clr, &c, &im, &bm);
        verdict[e] = ok ? 1 : 0;
        if (clearance) clearance[e] = clr;
        if (nchk) nchk[e] = c;
        if (int_margin) int_margin[e] = im;
        if (bound_margin) bound_margin[e] = bm;
    }
}

// Continuous verdicts and exact clearances of point-robot edges.
int orc_check_edges_continuous(const orc_problem* prob, int n, const double* qa, const double* ta,
                               const double* qb, const double* tb, unsigned char* verdict, double* clearance) {
    Problem P = to_problem(prob);
    if (P.arm) return -1;
    int d = P.dof;
    for (int e = 0; e < n; ++e) {
        double clr;
        bool ok = edge_free_continuous(P, qa + (size_t)e * d, ta[e], qb + (size_t)e * d, tb[e], &clr);
        verdict[e] = ok ? 1 : 0;
        if (clearance) clearance[e] = clr;
    }
    return 0;
}

// Interval-root partition from explicit grid flags (k = kmin..kmin+nk-1).
// Outputs: uniform lower bounds and width; pieces [n][3] (lo, hi, group).
int orc_interval_partition(double Lg, double H, double dt, int N, double U, long kmin, int nk,
                           const unsigned char* free_flags, double* uni_lo, double* uni_width,
                           double* pieces, int max_pieces) {
    IntervalAlloc A;
    A.Lg = Lg;
    A.H = H;
    A.dt = dt;
    A.N = N;
    std::vector<char> f(free_flags, free_flags + nk);
    if (nk > 0) build_windows(A, kmin, kmin + nk - 1, f.data());
    partition(A, U);
    for (int g = 0; g < N; ++g) uni_lo[g] = Lg + (double)g * A.width;
    *uni_width = A.width;
    int n = (int)A.pieces.size();
    for (int i = 0; i < n && i < max_pieces; ++i) {
        pieces[3 * i] = A.pieces[i].lo;
        pieces[3 * i + 1] = A.pieces[i].hi;
        pieces[3 * i + 2] = (double)A.pieces[i].group;
    }
    return n;
}

// Goal-time sample from an interval partition (for distribution tests).
double orc_interval_sample(double Lg, double H, double dt, int N, double U, long kmin, int nk,
                           const unsigned char* free_flags, int group, double u_coin, double u_pos,
                           double p_guided, int* guided) {
    IntervalAlloc A;
    A.Lg = Lg;
    A.H = H;
    A.dt = dt;
    A.N = N;
    std::vector<char> f(free_flags, free_flags + nk);
    if (nk > 0) build_windows(A, kmin, kmin + nk - 1, f.data());
    partition(A, U);
    bool g;
    double T = sample_goal_time(A, group, u_coin, u_pos, p_guided, &g);
    *guided = g ? 1 : 0;
    return T;
}

// Root-recycling update on its own: slots (T, has_root, active, gen) in/out.
// Grid: goal checks k = kmin..kmin+nk-1 with flags; dt grid spacing. Slot
// times must lie on the grid. Returns the number of replaced slots.
int orc_recycle_update(int N, double* T, int* has_root, int* active, int* gen, double U, long kmin, int nk,
                       const unsigned char* free_flags, double dt) {
    std::vector<Slot> slots(N);
    for (int i = 0; i < N; ++i) {
        slots[i].has_root = has_root[i] != 0;
        slots[i].active = active[i] != 0;
        slots[i].T = has_root[i] ? T[i] : kInf;
        slots[i].k = has_root[i] ? (long)std::llround(T[i] / dt) : -1;
        slots[i].gen = gen[i];
    }
    auto is_free = [&](long k) { return k >= kmin && k - kmin < nk && free_flags[k - kmin] != 0; };
    std::vector<int> rep = recycle_rule(slots, U, kmin, dt, is_free);
    for (int i = 0; i < N; ++i) {
        T[i] = slots[i].T;
        has_root[i] = slots[i].has_root;
        active[i] = slots[i].active;
        gen[i] = slots[i].gen;
    }
    return (int)rep.size();
}

struct orc_result {
    Result R;
};

// Learned-branch draws of worker w at iteration k (pins): learned flag,
// waypoint index, q_r [dof] (plain uniforms overwritten when learned), the
// mixture goal time T_l (interval root only: NaN when not learned).
int orc_learned_sample(const double* y, const double* qlo, const double* qhi, const double* qs, const double* qg,
                       int dof, double H, unsigned long long seed, unsigned problem_id, unsigned k, unsigned w,
                       int* wp_index, double* qr, double* Tl) {
    std::vector<double> lo(qlo, qlo + dof), hi(qhi, qhi + dof), s0(qs, qs + dof), g0(qg, qg + dof);
    Learned L;
    build_learned(L, y, lo, hi, s0, g0, dof, H);
    Draws dr;
    dr.fill(seed, problem_id, k, w, 17);
    const bool lrn = (dr.raw[12] >> 8) < kThrLearned;
    for (int j = 0; j < dof; ++j) qr[j] = lo[j] + dr.u(4 + j) * (hi[j] - lo[j]);
    *wp_index = dr.group(13, 16);
    *Tl = std::nan("");
    if (lrn) {
        learned_q(L, dr, lo, hi, dof, qr);
        double cm;
        *Tl = learned_T(L, dr, &cm);
    }
    return lrn ? 1 : 0;
}

int orc_plan(const orc_problem* prob, const orc_params* p, orc_result** out) {
    Problem P = to_problem(prob);
    // A query of a goal sequence starts at absolute time t_offset: its local
    // time 0 sees the obstacle trajectories shifted by t_offset (Sec. "Problem
    // Formulation").
    for (size_t i = 0; i < P.way.size(); i += 4) P.way[i] -= p->t_offset;
    Params prm;
    prm.variant = p->variant;
    prm.N = p->n_roots;
    prm.W = p->workers;
    prm.max_iters = p->max_iters;
    prm.eta = p->eta;
    prm.res = p->res;
    prm.dt = p->dt;
    prm.p_new = p->p_new;
    prm.p_guided = p->p_guided;
    prm.H = p->H;
    prm.seed = p->seed;
    prm.problem_id = p->problem_id;
    if (p->flag_tol > 0) prm.flag_tol = p->flag_tol;
    if (p->flag_clear > 0) prm.flag_clear = p->flag_clear;
    if (p->learned) {
        if (!p->proposal) return -1;
        prm.proposal = p->proposal;
    }
    if (p->continuous) {
        if (P.arm) return -1;
        prm.continuous = 1;
    }
    prm.follow_rec = p->follow_rec;
    prm.follow_iters = p->follow_iters;
    prm.follow_grid = p->follow_grid;
    prm.follow_nk = p->follow_nk;
    Planner pl(P, prm);
    orc_result* r = new orc_result;
    r->R = pl.run();
    *out = r;
    return r->R.status;
}

// summary: [U, C, iters, first_iter, ext_checked, bridge_checked, root_checked,
//           inserted, path_len, n_fwd, n_trees, status]
void orc_result_summary(const orc_result* r, double* s) {
    const Result& R = r->R;
    s[0] = R.U;
    s[1] = R.C;
    s[2] = R.iters;
    s[3] = R.first_iter;
    s[4] = (double)R.ext_checked;
    s[5] = (double)R.bridge_checked;
    s[6] = (double)R.root_checked;
    s[7] = (double)R.inserted;
    s[8] = R.dof > 0 ? (double)(R.path.size() / (R.dof + 1)) : 0.0;
    s[9] = (double)R.fwd.size();
    s[10] = (double)R.trees.size();
    s[11] = R.status;
}

void orc_result_path(const orc_result* r, double* path) {
    std::memcpy(path, r->R.path.data(), r->R.path.size() * sizeof(double));
}

// arena -1: forward tree; arena i >= 0: backward group / slot i.
int orc_result_arena_size(const orc_result* r, int arena) {
    if (arena < 0) return (int)r->R.fwd.size();
    if (arena >= (int)r->R.seg.size()) return 0;
    return (int)r->R.seg[arena].size();
}

void orc_result_arena(const orc_result* r, int arena, double* x, int* parent, double* troot, double* cost,
                      int* tree, int* iter) {
    const std::vector<Node>& A = arena < 0 ? r->R.fwd : r->R.seg[arena];
    int d = r->R.dof;
    for (size_t i = 0; i < A.size(); ++i) {
        for (int j = 0; j < d; ++j) x[i * (d + 1) + j] = A[i].q[j];
        x[i * (d + 1) + d] = A[i].t;
        parent[i] = A[i].parent;
        troot[i] = A[i].troot;
        cost[i] = A[i].cost;
        tree[i] = A[i].tree;
        iter[i] = A[i].iter;
    }
}

// Per-iteration U, smallest decision margin and smallest |clearance|.
void orc_result_history(const orc_result* r, double* U, double* margin, double* clear) {
    size_t n = r->R.U_hist.size();
    for (size_t i = 0; i < n; ++i) {
        U[i] = r->R.U_hist[i];
        margin[i] = r->R.margin_hist[i];
        clear[i] = r->R.clear_hist[i];
    }
}

// NN under rho_sigma over explicit nodes x [n][d+1] (q..., t), tie: lowest index.
int orc_nn_spacetime(int n, int d, const double* x, const double* troot, int filter, double U, const double* qr,
                     double tr, int sigma, double vmax, double* rho) {
    std::vector<Node> A(n);
    for (int i = 0; i < n; ++i) {
        A[i].q.assign(x + (size_t)i * (d + 1), x + (size_t)i * (d + 1) + d);
        A[i].t = x[(size_t)i * (d + 1) + d];
        A[i].troot = troot ? troot[i] : 0.0;
    }
    Margin M;
    return nn_spacetime(A, n, filter != 0, U, qr, tr, sigma, d, vmax, rho, M, 1e-5);
}

void orc_result_margin_types(const orc_result* r, double* out) {
    std::memcpy(out, r->R.margin_types.data(), r->R.margin_types.size() * sizeof(double));
}

// Slots (root recycling): T, has_root, active, gen per slot; trees (interval): group, T.
void orc_result_slots(const orc_result* r, double* T, int* has_root, int* active, int* gen) {
    for (size_t i = 0; i < r->R.slots.size(); ++i) {
        T[i] = r->R.slots[i].T;
        has_root[i] = r->R.slots[i].has_root;
        active[i] = r->R.slots[i].active;
        gen[i] = r->R.slots[i].gen;
    }
}

void orc_result_trees(const orc_result* r, int* group, double* T) {
    for (size_t i = 0; i < r->R.trees.size(); ++i) {
        group[i] = r->R.trees[i].group;
        T[i] = r->R.trees[i].T;
    }
}

int orc_result_goal_grid(const orc_result* r, long* kmin, double* clearance, int cap) {
    *kmin = r->R.goal_kmin;
    int n = (int)r->R.goal_clearance.size();
    for (int i = 0; i < n && i < cap; ++i) clearance[i] = r->R.goal_clearance[i];
    return n;
}

void orc_result_incumbent(const orc_result* r, int* f, int* s, int* b) {
    *f = r->R.inc_fwd;
    *s = r->R.inc_seg;
    *b = r->R.inc_bwd;
}

// Per-iteration incumbent length C (after the iteration's publish).
void orc_result_C_history(const orc_result* r, double* C) {
    std::memcpy(C, r->R.C_hist.data(), r->R.C_hist.size() * sizeof(double));
}

// Decision records [iters][W][10] and (T, t_r, window lo, window hi) [iters][W][4].
void orc_result_trace(const orc_result* r, int* rec, double* d) {
    if (rec) std::memcpy(rec, r->R.trace.data(), r->R.trace.size() * sizeof(int));
    if (d) std::memcpy(d, r->R.trace_d.data(), r->R.trace_d.size() * sizeof(double));
}

// Follow mode: per decision kind the adopted and differing counts
// [kinds], and the number of unflagged mismatches; unflagged [n][3] =
// (iteration, worker, kind) (iteration -1: goal-grid entry `worker`).
int orc_result_follow(const orc_result* r, long long* followed, long long* flagged_diff, int* unflagged, int cap) {
    for (int i = 0; i < kKinds; ++i) {
        if (followed) followed[i] = r->R.followed[i];
        if (flagged_diff) flagged_diff[i] = r->R.flagged_diff[i];
    }
    const int n = (int)(r->R.unflagged.size() / 3);
    if (unflagged)
        for (int i = 0; i < 3 * std::min(n, cap); ++i) unflagged[i] = r->R.unflagged[i];
    return n;
}

int orc_follow_kinds(void) { return kKinds; }

// Configuration-distance NN (root recycling) over explicit configurations
// x [n][d]; tie: lowest index. Returns the index (-1 if n == 0) and D.
int orc_nn_config(int n, int d, const double* x, const double* qr, double* D) {
    std::vector<Node> A(n);
    for (int i = 0; i < n; ++i) A[i].q.assign(x + (size_t)i * d, x + (size_t)i * d + d);
    Margin M;
    return nn_config(A, n, qr, d, D, M);
}

// Publish reduction over n successful bridges (U, C, worker): index of the
// lexicographic minimum (-1 if n == 0).
int orc_publish_winner(int n, const double* U, const double* C, const int* w) {
    int b = -1;
    for (int i = 0; i < n; ++i)
        if (b < 0 || publish_before(U[i], C[i], w[i], U[b], C[b], w[b])) b = i;
    return b;
}

// One bridge step of an inserted node a = (q_a, t_a) with root time troot_a
// and cost cost_a: rank the candidates, test the top one for improving
// (U0, C0) and validate only that one. forward: a is a forward node and the
// candidates are backward nodes of groups seg[i] (non-decreasing); else the
// candidates are forward nodes. Candidate rows x [n][d+1] (q, t), root times,
// costs. out[0..3] = (candidate group or -1, index within its group, improves,
// edges validated); out_d[0..1] = (U, C) of the candidate. Returns 1 if the
// bridge is collision-free and improves, else 0.
int orc_bridge(const orc_problem* prob, const double* qa, double ta, double troot_a, double cost_a, int forward,
               int n, const double* x, const double* troot, const double* cost, const int* seg, double U0,
               double C0, double res, int* out, double* out_d) {
    Problem P = to_problem(prob);
    const int d = P.dof;
    Node a;
    a.q.assign(qa, qa + d);
    a.t = ta;
    a.troot = troot_a;
    a.cost = cost_a;
    std::vector<std::vector<Node>> segs;
    std::vector<int> seg_n;
    std::vector<Node> fwd;
    std::vector<int> local(n, 0);
    for (int i = 0; i < n; ++i) {
        Node v;
        v.q.assign(x + (size_t)i * (d + 1), x + (size_t)i * (d + 1) + d);
        v.t = x[(size_t)i * (d + 1) + d];
        v.troot = troot[i];
        v.cost = cost[i];
        if (forward) {
            const int s = seg[i];
            if (s < 0) return -1;
            if ((int)segs.size() <= s) segs.resize(s + 1);
            local[i] = (int)segs[s].size();
            segs[s].push_back(v);
        } else {
            fwd.push_back(v);
        }
    }
    for (const auto& sg : segs) seg_n.push_back((int)sg.size());
    BridgeCand c = bridge_rank(a, forward != 0, segs, seg_n, fwd, (int)fwd.size(), U0, d, P.vmax, 1e-5);
    out[0] = c.s;
    out[1] = c.i;
    out[2] = 0;
    out[3] = 0;
    out_d[0] = out_d[1] = kInf;
    if (c.i < 0) return 0;
    const Node& b = forward ? segs[c.s][c.i] : fwd[c.i];
    const Node& fn = forward ? a : b;
    const Node& bn = forward ? b : a;
    const double Uc = bn.troot;
    const double Cc = fn.cost + dist(fn.q.data(), bn.q.data(), d) + bn.cost;
    out_d[0] = Uc;
    out_d[1] = Cc;
    const bool improves = (Uc < U0) || (Uc == U0 && Cc < C0);
    out[2] = improves ? 1 : 0;
    if (!improves) return 0;
    double clr;
    int cnt;
    const bool ok = edge_free(P, fn.q.data(), fn.t, bn.q.data(), bn.t, res, &clr, &cnt, nullptr);
    out[3] = 1;
    return ok ? 1 : 0;
}

void orc_result_free(orc_result* r) { delete r; }

}  // extern "C"
