// transport.cu -- event-based fixed-source transport kernels (compiled with
// --fmad=false: FP64 expressions are evaluated as written, except the few
// fused multiply-adds and stored reciprocals named where they are used, which
// move values by an ulp or so; per-history decisions stay those of a
// sequential FP64 evaluation in every history-matched test).
//
// Event-based mode (Sec. 5.1 of the paper): a buffer of particles in flight is
// advanced one event at a time, one kernel per event type over all particles
// that need it; dead slots are refilled from the remaining histories after
// every iteration.  One iteration here is
//     refill -> [bin XS queue] -> lookup -> advance (flight, tally, surface
//     crossing) -> [bin collision queue] -> collide -> bookkeeping
// In queueless mode each kernel visits every slot and returns early for
// particles that do not need its event; in queued mode the kernels visit
// device-built index queues (warp-ballot compaction) and never read a slot
// they do not need.  Queue sizes stay on the device: no host round trip per
// kernel.
//
// Fullest-queue mode (the paper's queued policy, Sec. 5.1, with the choice
// made on the device instead of the host): every live particle sits in
// exactly one state queue -- needs a lookup, needs a flight, needs a
// collision -- and free slots sit in a fourth.  One step is
//     refill (drains the free-slot queue) -> select -> [bin] -> the event
//     kernel of the queue the select kernel found fullest
// The queues are rings over the slot count with 64-bit head/tail positions;
// the flight queue has two rings, so that the flight kernel, whose surviving
// particles re-enter the flight queue, never appends into the ring it reads.
// No kernel appends to the ring it consumes, and a slot is in at most one
// ring, so a ring never holds more than the slot count.
//
// Tally scores are reduced within each warp (lanes that hit the same tally
// cell are found with __match_any_sync and summed with shuffles) and a single
// FP64 atomicAdd per distinct cell is issued.
#include "kernels.h"
#include "xs_exact.cuh"

// Flight geometry with fused multiply-adds (the move x + d u and the
// cylinder quadratic): values within an ulp of the as-written expressions,
// measured 1 % faster on the lattice; history-matched tests still reproduce
// every collision count.
#ifndef MCX_TRANSPORT_GEOM_FMA
#define MCX_TRANSPORT_GEOM_FMA 1
#endif
// Fewer FP64 divisions in direction sampling: one reciprocal for the
// azimuth's two quotients, a / b once in the rotation, and the lab cosine
// from a reciprocal square root (each within an ulp or two): 1.7 % faster on
// the lattice, collision counts still history-matched.
#ifndef MCX_TRANSPORT_RECIP_DIR
#define MCX_TRANSPORT_RECIP_DIR 1
#endif
// Elastic kinematics with the stored 1 / (A + 1)^2 and the rotation from one
// reciprocal square root (rotate_raw): FP64 divisions and square roots are
// multi-instruction sequences on B300's 1/64-rate FP64 pipe.
#ifndef MCX_TRANSPORT_KINEMATICS
#define MCX_TRANSPORT_KINEMATICS 1
#endif
// A flight divides once: the surface candidates and the collision distance
// are compared as quotients by cross-multiplication (surface_candidate).
#ifndef MCX_TRANSPORT_ONE_DIV
#define MCX_TRANSPORT_ONE_DIV 1
#endif
// The flight length -ln(xi) from a table-driven logarithm (neg_log_uniform)
// instead of the library's.
#ifndef MCX_TRANSPORT_TABLE_LOG
#define MCX_TRANSPORT_TABLE_LOG 1
#endif
// The lookup kernel takes a warp per particle when the queue holds at most
// one particle per warp of its grid (macro_transport_warp).
#ifndef MCX_TRANSPORT_WARP_TAIL
#define MCX_TRANSPORT_WARP_TAIL 1
#endif

namespace mcx {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr double INF = __builtin_huge_val();

enum { S_NONE = 0, S_ZTOP, S_ZBOT, S_CYL, S_XLO, S_XHI, S_YLO, S_YHI };
constexpr int MAX_AZIMUTH_TRIES = 64;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ unsigned lanes_below() { return (1u << lane_id()) - 1u; }

// Warp-aggregated append: every lane of the (converged) warp calls it; each
// lane with `want` receives a distinct slot of the queue behind `counter`.
__device__ __forceinline__ int warp_append(int* counter, bool want)
{
    const unsigned b = __ballot_sync(FULL, want);
    if (b == 0u) return -1;
    const int leader = __ffs(b) - 1;
    int base = 0;
    if (lane_id() == leader) base = atomicAdd(counter, __popc(b));
    base = __shfl_sync(FULL, base, leader);
    return want ? base + __popc(b & lanes_below()) : -1;
}

// Bounds-checked builds: a particle slot read from an event queue, and an
// append position, outside [0, cap) stop the run (MCX_ERR_BOUNDS) and are
// replaced by slot 0 / not written.
__device__ __forceinline__ int64_t checked_slot(int64_t slot, const Particles& P, RunCtl* ctl)
{
#if MCX_BOUNDS_CHECK
    if (!MCX_IN_BOUNDS(slot >= 0 && slot < P.cap, BC_SLOT, slot)) {
        atomicCAS(&ctl->error, 0, MCX_ERR_BOUNDS);
        return 0;
    }
#endif
    return slot;
}

__device__ __forceinline__ void queue_put(int32_t* q, int64_t pos, int64_t slot, const Particles& P, RunCtl* ctl)
{
#if MCX_BOUNDS_CHECK
    if (!MCX_IN_BOUNDS(pos >= 0 && pos < P.cap, BC_QUEUE, pos)) {
        atomicCAS(&ctl->error, 0, MCX_ERR_BOUNDS);
        return;
    }
#endif
    q[pos] = (int32_t)slot;
}

// Where an event kernel takes its particles from: every slot (list == null),
// a compacted list, or a segment of a ring (positions wrap at `wrap`).
struct Src {
    const int32_t* list;
    int64_t n;
    int64_t start;
    int64_t wrap;
};

__device__ __forceinline__ Src all_slots(const Particles& P) { return Src{nullptr, P.cap, 0, 0}; }
__device__ __forceinline__ Src plain_list(const int32_t* list, int64_t n)
{
    return Src{list, n, 0, INT64_MAX};
}

__device__ __forceinline__ int64_t src_at(const Src& s, int64_t i)
{
    if (!s.list) return i;
    int64_t k = s.start + i;       // start < wrap and n <= wrap: one fold suffices
    if (k >= s.wrap) k -= s.wrap;
    return s.list[k];
}

__device__ __forceinline__ int32_t* ring_base(const Particles& P, int r)
{
    switch (r) {
    case RQ_XS: return P.q_xs[0];
    case RQ_ADV0: return P.q_adv[0];
    case RQ_ADV1: return P.q_adv[1];
    case RQ_COLL: return P.q_coll;
    default: return P.q_dead[0];
    }
}

// The segment the select kernel handed to this step's event kernel.
__device__ __forceinline__ Src ring_segment(const Particles& P, const RunCtl* ctl)
{
    return Src{ring_base(P, ctl->sel_ring), (int64_t)(ctl->sel_end - ctl->sel_begin),
               (int64_t)(ctl->sel_begin % (unsigned long long)P.cap), P.cap};
}

// Warp-aggregated append to ring r (every lane of the converged warp calls it).
__device__ __forceinline__ void ring_push(const Particles& P, RunCtl* ctl, int r, bool want, int64_t slot)
{
    const unsigned b = __ballot_sync(FULL, want);
    if (b == 0u) return;
    const int leader = __ffs(b) - 1;
    unsigned long long base = 0ull;
    if (lane_id() == leader) base = atomicAdd(&ctl->rq_tail[r], (unsigned long long)__popc(b));
    base = __shfl_sync(FULL, base, leader);
    if (want) {
        const unsigned long long pos = (base + __popc(b & lanes_below())) % (unsigned long long)P.cap;
        ring_base(P, r)[pos] = (int32_t)slot;
    }
}

// Sum of v over the lanes with `on`, added to *a with one atomic (every lane
// of the converged warp calls it).
__device__ __forceinline__ void warp_add(double* a, double v, bool on)
{
    const unsigned m = __ballot_sync(FULL, on);
    if (m == 0u) return;
    double s = on ? v : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if (lane_id() == __ffs(m) - 1) atomicAdd(a, s);
}

#ifndef MCX_TALLY_TREE
#define MCX_TALLY_TREE 1
#endif
#ifndef MCX_TRANSPORT_CONVERGED
#define MCX_TRANSPORT_CONVERGED 1
#endif
#ifndef MCX_LOOKUP_CLAIM
#define MCX_LOOKUP_CLAIM 1
#endif
// Sign tests of a non-NaN double on its bit pattern: the answers of the
// comparisons with zero (-0.0 included), on the integer pipes instead of
// B300's FP64 pipe, which also executes FP64 comparisons and limits the flight.
#ifndef MCX_TRANSPORT_INT_SIGN
#define MCX_TRANSPORT_INT_SIGN 1
#endif
#if MCX_TRANSPORT_INT_SIGN
__device__ __forceinline__ bool gt0(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool lt0(double x)
{
    const long long b = __double_as_longlong(x);
    return b < 0 && b != (long long)0x8000000000000000ull;
}
__device__ __forceinline__ bool ge0(double x)
{
    const long long b = __double_as_longlong(x);
    return b >= 0 || b == (long long)0x8000000000000000ull;
}
__device__ __forceinline__ bool ne0(double x) { return ((unsigned long long)__double_as_longlong(x) << 1) != 0ull; }
#else
__device__ __forceinline__ bool gt0(double x) { return x > 0.0; }
__device__ __forceinline__ bool lt0(double x) { return x < 0.0; }
__device__ __forceinline__ bool ge0(double x) { return x >= 0.0; }
__device__ __forceinline__ bool ne0(double x) { return x != 0.0; }
#endif

// Lane holding the r-th (from 0) set bit of m; requires r < popc(m).
__device__ __forceinline__ int nth_lane(unsigned m, int r)
{
    int pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const int c = __popc(m & ((1u << w) - 1u));
        if (r >= c) {
            r -= c;
            m >>= w;
            pos += w;
        }
    }
    return pos;
}

// Sums of v[0..NV) over the lanes of each lane's group `grp` (the lanes with
// an equal key, from __match_any_sync), left in the group's lowest lane.
// Every lane of the converged warp calls it.  A shift-down tree over each
// group's lanes in rank order: ceil(log2(largest group)) steps of one FP64
// add per value, where summing the group's lanes one by one would take as
// many steps as the largest group has lanes.
template <int NV>
__device__ __forceinline__ void group_sum(unsigned grp, double (&v)[NV])
{
    const int rank = __popc(grp & lanes_below());
    const int size = __popc(grp);
    const int most = (int)__reduce_max_sync(FULL, (unsigned)size);
    for (int o = 1; o < most; o <<= 1) {
        const bool has = rank + o < size;
        const int src = has ? nth_lane(grp, rank + o) : lane_id();
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const double w = __shfl_sync(FULL, v[k], src);
            if (has) v[k] += w;
        }
    }
}

// -ln x for a uniform x in [2^-53, 1) (uniform_at's range), by Tang's
// table-driven method (P. T. P. Tang, ACM Trans. Math. Softw. 16, 378,
// 1990): x = 2^-t (F + f) with F = 1 + j/256 the leading 8 bits of the
// mantissa (so f = m - F is exact), and -ln x = t ln 2 - ln F - ln(1 + r),
// r = f / F < 2^-8, the last from its Taylor series to r^6 (remainder below
// 2^-59).  The table holds ln F_j, 1 / F_j and t ln 2, computed on the device
// with the library's logarithm and division.  About ten FP64 operations; the
// error is an ulp or two of max(1, -ln x) -- like the library's against the
// host's, not relative near x = 1 where -ln x is tiny (a flight of ~1e-16
// cm may come out a few 1e-17 cm longer or shorter).
constexpr int kNlN = 256;                     // table intervals of the mantissa
constexpr int kNlSize = 2 * kNlN + 64;        // ln F_j, 1 / F_j, t ln 2 (t < 64)
__device__ double g_nlog[kNlSize];

__global__ void k_init_nlog()
{
    for (int i = threadIdx.x; i < kNlSize; i += blockDim.x) {
        double v;
        if (i < kNlN) v = log(1.0 + i / 256.0);
        else if (i < 2 * kNlN) v = 1.0 / (1.0 + (i - kNlN) / 256.0);
        else v = log(ldexp(1.0, i - 2 * kNlN));
        g_nlog[i] = v;
    }
}

__device__ __forceinline__ double neg_log_uniform(double x)
{
#if MCX_TRANSPORT_TABLE_LOG
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int t = 1023 - (int)(b >> 52);                  // 1 .. 53 for x in [2^-53, 1)
    const uint64_t top = b & 0x000FF00000000000ull;       // leading 8 mantissa bits
    const int j = (int)(top >> 44);
    const double m = __longlong_as_double((long long)((b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull));
    const double F = __longlong_as_double((long long)(top | 0x3FF0000000000000ull));
    const double r = (m - F) * __ldg(&g_nlog[kNlN + j]);
    double q = fma(r, -1.0 / 6.0, 0.2);
    q = fma(r, q, -0.25);
    q = fma(r, q, 1.0 / 3.0);
    q = fma(r, q, -0.5);
    q = fma(r, q, 1.0);
    return (__ldg(&g_nlog[2 * kNlN + t]) - __ldg(&g_nlog[j])) - r * q;
#else
    return -log(x);
#endif
}

#ifndef MCX_SIGNED_UNIFORM
#define MCX_SIGNED_UNIFORM 1
#endif
// 2 u - 1 for u = uniform_at(key, hist, n), exactly: u = (2k + 1) 2^-53 makes
// 2u - 1 = (2k + 1 - 2^52) 2^-52, an odd integer below 2^52 in magnitude
// times 2^-52, which the FP64 multiply and subtract reproduce without
// rounding; built here from that integer's bits as uniform_at builds u.
__device__ __forceinline__ double uniform_signed(uint2 key, uint64_t hist, uint32_t n)
{
#if MCX_SIGNED_UNIFORM
    const uint4 w = philox4x32_10(make_uint4(n >> 1, (uint32_t)hist, (uint32_t)(hist >> 32), 0u), key);
    const uint32_t a = (n & 1u) ? w.z : w.x;
    const uint32_t b = (n & 1u) ? w.w : w.y;
    const uint64_t k = ((uint64_t)(a >> 6) << 26) | (uint64_t)(b >> 6);
    const int64_t N = (int64_t)(2 * k + 1) - (int64_t)(1ull << 52);
    const uint64_t sign = N < 0 ? 0x8000000000000000ull : 0ull;
    const uint64_t M = (uint64_t)(N < 0 ? -N : N);   // odd, 1 <= M < 2^52
    const int p = 63 - __clzll((long long)M);
    const uint64_t mant = (M << (52 - p)) & 0x000FFFFFFFFFFFFFull;
    return __longlong_as_double((long long)(sign | ((uint64_t)(p - 52 + 1023) << 52) | mant));
#else
    return 2.0 * uniform_at(key, hist, n) - 1.0;
#endif
}

// Azimuth (cos phi, sin phi) by rejection on pairs (2u-1, 2u-1) inside the
// unit disc.
__device__ __forceinline__ void azimuth(uint2 key, uint64_t h, uint32_t& n, double& c, double& s)
{
    for (int t = 0; t < MAX_AZIMUTH_TRIES; ++t) {
        const double a = uniform_signed(key, h, n);
        const double b = uniform_signed(key, h, n + 1);
        n += 2;
        const double rho = a * a + b * b;
        if (rho > 0.0 && rho <= 1.0) {
#if MCX_TRANSPORT_RECIP_DIR
            const double r = 1.0 / rho;
            c = (a * a - b * b) * r;
            s = (2.0 * a * b) * r;
#else
            c = (a * a - b * b) / rho;
            s = 2.0 * a * b / rho;
#endif
            return;
        }
    }
    c = 1.0;
    s = 0.0;
}

// The same draws as azimuth, unnormalised: (a^2 - b^2, 2 a b) = rho (cos phi,
// sin phi) and rho, so that the rotation can fold 1 / rho into its one
// reciprocal square root.
__device__ __forceinline__ void azimuth_raw(uint2 key, uint64_t h, uint32_t& n, double& c, double& s,
                                           double& rho)
{
    for (int t = 0; t < MAX_AZIMUTH_TRIES; ++t) {
        const double a = uniform_signed(key, h, n);
        const double b = uniform_signed(key, h, n + 1);
        n += 2;
        const double r = a * a + b * b;
        if (gt0(r) && r <= 1.0) {
            c = a * a - b * b;
            s = 2.0 * a * b;
            rho = r;
            return;
        }
    }
    c = 1.0;
    s = 0.0;
    rho = 1.0;
}

// Fission-spectrum energy: the Maxwellian sqrt(E) exp(-E/T), a Gamma(3/2, T)
// variate, as a Gamma(1) plus a Gamma(1/2) variate: E = -T (ln xi1 +
// ln xi2 cos^2 phi), phi uniform (the square of a Box-Muller normal;
// Everett and Cashwell's sampler, rule C64), cos phi from the disc rejection.
__device__ __forceinline__ double fission_energy(uint2 key, uint64_t h, uint32_t& n, double T)
{
    const double xi1 = uniform_at(key, h, n);
    const double xi2 = uniform_at(key, h, n + 1);
    n += 2;
    double c, s;
    azimuth(key, h, n, c, s);
    return -T * (log(xi1) + (c * c) * log(xi2));
}


struct State {
    double x, y, z, u, v, w;
    int32_t ci, cj, inpin;
};

#if !MCX_TRANSPORT_ONE_DIV
// Distance to the nearest surface along the flight.  Candidates are compared
// in a fixed order with strict '<' (earlier candidates win ties).
__device__ double surface_distance(const ProblemDev& pd, const State& q, int& surf)
{
    double d = INF;
    surf = S_NONE;
    if (pd.geometry == MCX_GEOM_INFINITE) return d;
    if (pd.geometry == MCX_GEOM_SLAB) {
        if (q.u > 0.0) {
            d = (pd.slab_length - q.x) / q.u;
            surf = S_XHI;
        } else if (q.u < 0.0) {
            d = (0.0 - q.x) / q.u;
            surf = S_XLO;
        }
        if (d < 0.0) d = 0.0;
        return d;
    }
    if (q.w > 0.0) {
        d = (pd.height - q.z) / q.w;
        surf = S_ZTOP;
    } else if (q.w < 0.0) {
        d = (0.0 - q.z) / q.w;
        surf = S_ZBOT;
    }
    const double cx = __ldg(pd.lat_centre + q.ci);
    const double cy = __ldg(pd.lat_centre + q.cj);
    const double dx = q.x - cx, dy = q.y - cy;
#if MCX_TRANSPORT_GEOM_FMA
    const double a = fma(q.u, q.u, q.v * q.v);
    const double k = fma(dx, q.u, dy * q.v);
    const double c = fma(dx, dx, fma(dy, dy, -(pd.radius * pd.radius)));
#else
    const double a = q.u * q.u + q.v * q.v;
    const double k = dx * q.u + dy * q.v;
    const double c = dx * dx + dy * dy - pd.radius * pd.radius;
#endif
    double dc = INF;
    if (q.inpin) {
        if (a > 0.0) {
#if MCX_TRANSPORT_GEOM_FMA
            double disc = fma(k, k, -(a * c));
#else
            double disc = k * k - a * c;
#endif
            if (disc < 0.0) disc = 0.0;
            dc = (-k + sqrt(disc)) / a;
        }
    } else if (a > 0.0 && k < 0.0) {
#if MCX_TRANSPORT_GEOM_FMA
        const double disc = fma(k, k, -(a * c));
#else
        const double disc = k * k - a * c;
#endif
        if (disc >= 0.0) dc = (-k - sqrt(disc)) / a;
    }
    if (dc < d) {
        d = dc;
        surf = S_CYL;
    }
    if (!q.inpin) {
        const double xl = __ldg(pd.lat_plane + q.ci);
        const double xh = __ldg(pd.lat_plane + q.ci + 1);
        const double yl = __ldg(pd.lat_plane + q.cj);
        const double yh = __ldg(pd.lat_plane + q.cj + 1);
        if (q.u > 0.0) {
            const double t = (xh - q.x) / q.u;
            if (t < d) { d = t; surf = S_XHI; }
        } else if (q.u < 0.0) {
            const double t = (xl - q.x) / q.u;
            if (t < d) { d = t; surf = S_XLO; }
        }
        if (q.v > 0.0) {
            const double t = (yh - q.y) / q.v;
            if (t < d) { d = t; surf = S_YHI; }
        } else if (q.v < 0.0) {
            const double t = (yl - q.y) / q.v;
            if (t < d) { d = t; surf = S_YLO; }
        }
    }
    if (d < 0.0) d = 0.0;
    return d;
}
#endif

// The same candidates as surface_distance, in the same order and with the
// same strict '<' between them, each kept as a quotient t = num / den with
// den > 0 and compared by cross-multiplication (t1 < t2 iff num1 den2 <
// num2 den1), so that a flight divides once, for the distance it takes.
// Returns den = 0 when no surface is ahead.
__device__ void surface_candidate(const ProblemDev& pd, const State& q, int& surf, double& num, double& den)
{
    num = 0.0;
    den = 0.0;
    surf = S_NONE;
    auto offer = [&](double n, double m, int s) {
        if (!ne0(den) || n * den < num * m) {
            num = n;
            den = m;
            surf = s;
        }
    };
    if (pd.geometry == MCX_GEOM_INFINITE) return;
    if (pd.geometry == MCX_GEOM_SLAB) {
        if (q.u > 0.0) offer(pd.slab_length - q.x, q.u, S_XHI);
        else if (q.u < 0.0) offer(q.x, -q.u, S_XLO);
        return;
    }
#if MCX_TRANSPORT_CONVERGED
    // Both directions of an axis, and both sides of the cylinder, in one
    // code path with selected operands (the same values as the branches
    // below): a warp that mixes directions or particles inside and outside
    // the pins issues each FP64 operation once instead of once per branch.
    {
        const bool up = gt0(q.w);
        if (ne0(q.w)) offer(up ? pd.height - q.z : q.z, up ? q.w : -q.w, up ? S_ZTOP : S_ZBOT);
    }
    const double cx = __ldg(pd.lat_centre + q.ci);
    const double cy = __ldg(pd.lat_centre + q.cj);
    const double dx = q.x - cx, dy = q.y - cy;
    const double a = fma(q.u, q.u, q.v * q.v);
    const double k = fma(dx, q.u, dy * q.v);
    const double c = fma(dx, dx, fma(dy, dy, -pd.radius2));
    {
        const double disc = fma(k, k, -(a * c));
        const double r = sqrt(lt0(disc) ? 0.0 : disc);
        if (gt0(a) && (q.inpin || (lt0(k) && ge0(disc)))) offer(q.inpin ? -k + r : -k - r, a, S_CYL);
    }
    if (!q.inpin) {
        const bool ux = gt0(q.u), uy = gt0(q.v);
        const double px = __ldg(pd.lat_plane + q.ci + (ux ? 1 : 0));
        const double py = __ldg(pd.lat_plane + q.cj + (uy ? 1 : 0));
        if (ne0(q.u)) offer(ux ? px - q.x : q.x - px, ux ? q.u : -q.u, ux ? S_XHI : S_XLO);
        if (ne0(q.v)) offer(uy ? py - q.y : q.y - py, uy ? q.v : -q.v, uy ? S_YHI : S_YLO);
    }
#else
    if (q.w > 0.0) offer(pd.height - q.z, q.w, S_ZTOP);
    else if (q.w < 0.0) offer(q.z, -q.w, S_ZBOT);
    const double cx = __ldg(pd.lat_centre + q.ci);
    const double cy = __ldg(pd.lat_centre + q.cj);
    const double dx = q.x - cx, dy = q.y - cy;
    const double a = fma(q.u, q.u, q.v * q.v);
    const double k = fma(dx, q.u, dy * q.v);
    const double c = fma(dx, dx, fma(dy, dy, -(pd.radius * pd.radius)));
    if (q.inpin) {
        if (a > 0.0) {
            double disc = fma(k, k, -(a * c));
            if (disc < 0.0) disc = 0.0;
            offer(-k + sqrt(disc), a, S_CYL);
        }
    } else if (a > 0.0 && k < 0.0) {
        const double disc = fma(k, k, -(a * c));
        if (disc >= 0.0) offer(-k - sqrt(disc), a, S_CYL);
    }
    if (!q.inpin) {
        if (q.u > 0.0) offer(__ldg(pd.lat_plane + q.ci + 1) - q.x, q.u, S_XHI);
        else if (q.u < 0.0) offer(q.x - __ldg(pd.lat_plane + q.ci), -q.u, S_XLO);
        if (q.v > 0.0) offer(__ldg(pd.lat_plane + q.cj + 1) - q.y, q.v, S_YHI);
        else if (q.v < 0.0) offer(q.y - __ldg(pd.lat_plane + q.cj), -q.v, S_YLO);
    }
#endif
}

// Logical crossing; returns the outcome if the particle leaves, else -1.
__device__ __forceinline__ int cross_surface(const ProblemDev& pd, State& q, int surf)
{
    const int32_t n = pd.lattice_n;
    switch (surf) {
    case S_ZTOP:
    case S_ZBOT:
        q.w = -q.w;
        return -1;
    case S_CYL:
        q.inpin = !q.inpin;
        return -1;
    case S_XHI:
        if (pd.geometry == MCX_GEOM_SLAB || q.ci == n - 1) return OUT_LEAK_XHI;
        q.ci += 1;
        return -1;
    case S_XLO:
        if (pd.geometry == MCX_GEOM_SLAB || q.ci == 0) return OUT_LEAK_OTHER;
        q.ci -= 1;
        return -1;
    case S_YHI:
        if (q.cj == n - 1) return OUT_LEAK_OTHER;
        q.cj += 1;
        return -1;
    case S_YLO:
        if (q.cj == 0) return OUT_LEAK_OTHER;
        q.cj -= 1;
        return -1;
    default:
        return OUT_LEAK_OTHER;
    }
}

__device__ __forceinline__ int32_t region_of(const ProblemDev& pd, const State& q)
{
    if (pd.geometry != MCX_GEOM_LATTICE) return 0;
    return q.inpin ? q.ci * pd.lattice_n + q.cj : pd.lattice_n * pd.lattice_n;
}

// rotate() with (c, s) = rho (cos phi, sin phi) unnormalised: with
// m = 1 - mu^2 and t = 1 - w0^2 (or 1 - v0^2), the factor sin(theta) /
// (sqrt(t) rho) the rotation needs is m / sqrt(m t rho^2) -- one reciprocal
// square root in place of two square roots and two divisions (the same
// rotation up to rounding).
__device__ __forceinline__ void rotate_raw(double& u, double& v, double& w, double mu, double c, double s,
                                           double rho)
{
    const double u0 = u, v0 = v, w0 = w;
    const double m = fma(-mu, mu, 1.0);
    const bool wz = fabs(w0) < 0.9999;
    const double t = wz ? fma(-w0, w0, 1.0) : fma(-v0, v0, 1.0);
    const double aq = gt0(m) ? m * rsqrt(m * t * (rho * rho)) : 0.0;
    if (wz) {
        u = fma(mu, u0, aq * fma(u0 * w0, c, -(v0 * s)));
        v = fma(mu, v0, aq * fma(v0 * w0, c, u0 * s));
        w = fma(mu, w0, -(aq * t * c));
    } else {
        u = fma(mu, u0, aq * fma(u0 * v0, c, w0 * s));
        v = fma(mu, v0, -(aq * t * c));
        w = fma(mu, w0, aq * fma(v0 * w0, c, -(u0 * s)));
    }
}

#if !MCX_TRANSPORT_KINEMATICS
__device__ __forceinline__ void rotate(double& u, double& v, double& w, double mu, double c, double s)
{
    const double u0 = u, v0 = v, w0 = w;
    const double a = sqrt(1.0 - mu * mu);
#if MCX_TRANSPORT_RECIP_DIR
    if (fabs(w0) < 0.9999) {
        const double b = sqrt(1.0 - w0 * w0);
        const double ab = a / b;
        u = mu * u0 + ab * (u0 * w0 * c - v0 * s);
        v = mu * v0 + ab * (v0 * w0 * c + u0 * s);
        w = mu * w0 - a * b * c;
    } else {
        const double b = sqrt(1.0 - v0 * v0);
        const double ab = a / b;
        u = mu * u0 + ab * (u0 * v0 * c + w0 * s);
        v = mu * v0 - a * b * c;
        w = mu * w0 + ab * (v0 * w0 * c - u0 * s);
    }
#else
    if (fabs(w0) < 0.9999) {
        const double b = sqrt(1.0 - w0 * w0);
        u = mu * u0 + a * (u0 * w0 * c - v0 * s) / b;
        v = mu * v0 + a * (v0 * w0 * c + u0 * s) / b;
        w = mu * w0 - a * b * c;
    } else {
        const double b = sqrt(1.0 - v0 * v0);
        u = mu * u0 + a * (u0 * v0 * c + w0 * s) / b;
        v = mu * v0 - a * b * c;
        w = mu * w0 + a * (v0 * w0 * c - u0 * s) / b;
    }
#endif
}
#endif

__device__ __forceinline__ int64_t batch_of(const ProblemDev& pd, int64_t h)
{
    return ((h - pd.tally_off) * (int64_t)pd.n_batches) / pd.n_hist_total;
}

// Map a work item to (problem, history).
__device__ __forceinline__ int problem_of_work(const int64_t* work_off, int n_prob, long long wk)
{
    int lo = 0, hi = n_prob - 1;  // largest p with work_off[p] <= wk
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (work_off[mid] <= wk) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Source particle of history h (lattice: centre of a uniformly chosen pin at
// mid-height; infinite medium: origin; both isotropic; slab: pencil along +x).
template <bool EIG>
__device__ void init_particle(const Particles& P, int64_t slot, const ProblemDev& pd,
                              int32_t pidx, int64_t h, int M)
{
    const uint2 key = pd.key;
    uint32_t n = 0;
    State q = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0, 0, 0};
    double E0 = pd.E0;
    if (EIG && pd.src) {
        // eigenvalue generation: start at the history's fission site,
        // isotropic, with a fission-spectrum energy
        const FissionSite site = pd.src[h - pd.first];
        const int32_t ln = pd.lattice_n > 0 ? pd.lattice_n : 1;
        q.x = site.x;
        q.y = site.y;
        q.z = site.z;
        q.ci = site.cell / ln;
        q.cj = site.cell % ln;
        q.inpin = site.inpin;
        const double mu = uniform_signed(key, h, n);
        n += 1;
        double c, s;
        azimuth(key, h, n, c, s);
        const double st = sqrt(1.0 - mu * mu);
        q.u = st * c;
        q.v = st * s;
        q.w = mu;
        E0 = fission_energy(key, h, n, pd.T_fission);
    } else if (pd.geometry == MCX_GEOM_SLAB) {
        q.u = 1.0;
    } else {
        if (pd.geometry == MCX_GEOM_LATTICE) {
            const int32_t ln = pd.lattice_n;
            const int64_t n2 = (int64_t)ln * ln;
            int64_t pin = (int64_t)(uniform_at(key, h, n) * (double)n2);
            n += 1;
            if (pin >= n2) pin = n2 - 1;
            q.ci = (int32_t)(pin / ln);
            q.cj = (int32_t)(pin % ln);
            q.x = __ldg(pd.lat_centre + q.ci);
            q.y = __ldg(pd.lat_centre + q.cj);
            q.z = 0.5 * pd.height;
            q.inpin = 1;
        }
        const double mu = uniform_signed(key, h, n);
        n += 1;
        double c, s;
        azimuth(key, h, n, c, s);
        const double st = sqrt(1.0 - mu * mu);
        q.u = st * c;
        q.v = st * s;
        q.w = mu;
    }
    P.x[slot] = q.x; P.y[slot] = q.y; P.z[slot] = q.z;
    P.u[slot] = q.u; P.v[slot] = q.v; P.w[slot] = q.w;
    P.E[slot] = E0;
    P.hist[slot] = h;
    if (EIG) P.nsite[slot] = 0u;
    P.rng_n[slot] = n;
    P.ncoll[slot] = 0u;
    P.cell[slot] = q.ci * (pd.lattice_n > 0 ? pd.lattice_n : 1) + q.cj;
    P.mat[slot] = __ldg(pd.region_material + region_of(pd, q));
    P.prob[slot] = pidx;
    P.flags[slot] = (uint8_t)(PF_ALIVE | PF_NEED_XS | (q.inpin ? PF_INPIN : 0));
    for (int mm = 0; mm < M; ++mm) P.W[(int64_t)mm * P.stride + slot] = 0.0;
}

__device__ __forceinline__ State load_state(const Particles& P, int64_t slot, int32_t ln)
{
    State q;
    q.x = P.x[slot]; q.y = P.y[slot]; q.z = P.z[slot];
    q.u = P.u[slot]; q.v = P.v[slot]; q.w = P.w[slot];
    const int32_t cell = P.cell[slot];
    const int32_t n = ln > 0 ? ln : 1;
    q.ci = cell / n;
    q.cj = cell % n;
    q.inpin = (P.flags[slot] & PF_INPIN) ? 1 : 0;
    return q;
}

// Deaths of this warp: outcome tallies (one atomic per distinct tally cell),
// derivative outcome tallies, per-history debug counts, slot release, alive
// count and (queued modes) the free-slot queue.  Every lane of the warp calls it.
template <bool EIG>
__device__ void finish_deaths(bool dies, int outcome, int64_t slot, int32_t pidx,
                              const ProblemDev* probs, const Particles& P, RunCtl* ctl, int M,
                              int mode, int par)
{
    const unsigned dm = __ballot_sync(FULL, dies);
    if (dm == 0u) return;
    const ProblemDev& pd = probs[pidx];
    int64_t h = 0, b = 0;
    double* a = nullptr;
    if (dies) {
        h = P.hist[slot];
        b = batch_of(pd, h);
        a = pd.outcome + b * N_OUT + outcome;
    }
    // lanes that do not die share the key 0, a group whose sums are not added
    const unsigned grp = __match_any_sync(FULL, dies ? (unsigned long long)a : 0ull);
    const bool lead = dies && lane_id() == __ffs(grp) - 1;
    if (lead) atomicAdd(a, (double)__popc(grp));
    for (int mm = 0; mm < M; ++mm) {
        double wv[1] = {dies ? P.W[(int64_t)mm * P.stride + slot] : 0.0};
        group_sum(grp, wv);
        if (lead) atomicAdd(pd.doutcome + (b * N_OUT + outcome) * M + mm, wv[0]);
    }
    if (dies) {
        if (pd.ncoll_debug) pd.ncoll_debug[h - pd.first] = P.ncoll[slot];
        if (EIG && pd.site_count) pd.site_count[h - pd.first] = P.nsite[slot];
        P.flags[slot] = 0;
    }
    if (lane_id() == 0) atomicSub(&ctl->n_alive, __popc(dm));
    if (mode == MCX_QUEUED) {
        const int pos = warp_append(&ctl->n_dead[par ^ 1], dies);
        if (dies) queue_put(P.q_dead[par ^ 1], pos, slot, P, ctl);
    } else if (mode == MCX_QUEUED_FULLEST) {
        ring_push(P, ctl, RQ_DEAD, dies, slot);
    }
}

// ------------------------------------------------------------------ kernels

__global__ void k_run_init(Particles P, RunCtl* ctl, long long total, int n_prob,
                           long long max_iters, int mode)
{
    const bool queued = mode != MCX_QUEUELESS;   // every slot starts in the free-slot queue
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.cap; i += stride) {
        P.flags[i] = 0;
        if (queued) P.q_dead[0][i] = (int32_t)i;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->next = 0ull;
        ctl->total = total;
        ctl->iters = 0;
        ctl->max_iters = max_iters;
        ctl->n_prob = n_prob;
        ctl->n_alive = 0;
        ctl->done = total > 0 ? 0 : 1;
        ctl->error = 0;
        ctl->parity = 0;
        for (int k = 0; k < 2; ++k) {
            ctl->n_xs[k] = 0;
            ctl->n_adv[k] = 0;
            ctl->n_dead[k] = 0;
        }
        ctl->n_dead[0] = queued ? (int)P.cap : 0;
        ctl->n_coll = 0;
        ctl->sorted = 0;
        ctl->sort_which = 0;
        ctl->lk_claim = 0ull;
        for (int r = 0; r < N_RQ; ++r) {
            ctl->rq_head[r] = 0ull;
            ctl->rq_tail[r] = 0ull;
        }
        ctl->rq_tail[RQ_DEAD] = mode == MCX_QUEUED_FULLEST ? (unsigned long long)P.cap : 0ull;
        ctl->adv_recv = 0;
        ctl->sel = -1;
        ctl->sel_ring = 0;
        ctl->sel_begin = 0ull;
        ctl->sel_end = 0ull;
        for (int e = 0; e < 3; ++e) ctl->sel_count[e] = 0;
        for (int e = 0; e < 4; ++e) ctl->ev_count[e] = 0;
    }
}

template <bool EIG>
__global__ void __launch_bounds__(1024) k_refill(LoopConfig c, Particles P, const ProblemDev* probs,
                                                 const int64_t* work_off, RunCtl* ctl)
{
    if (ctl->error || ctl->done) return;
    const bool queued = c.mode == MCX_QUEUED;
    const bool fq = c.mode == MCX_QUEUED_FULLEST;
    const int par = ctl->parity;
    const long long total = ctl->total;
    const int n_prob = ctl->n_prob;
    Src src = all_slots(P);
    if (queued) {
        src = plain_list(P.q_dead[par], ctl->n_dead[par]);
    } else if (fq) {
        // the whole free-slot ring; the select kernel that follows retires it
        const unsigned long long h0 = ctl->rq_head[RQ_DEAD], t0 = ctl->rq_tail[RQ_DEAD];
        src = Src{P.q_dead[0], (int64_t)(t0 - h0), (int64_t)(h0 % (unsigned long long)P.cap), P.cap};
        if (src.n > P.cap) {
            if (blockIdx.x == 0 && threadIdx.x == 0) ctl->error = MCX_ERR_STATE;
            return;
        }
    }
    const int64_t count = src.n;
    if ((long long)ctl->next >= total && (queued || fq)) {
        // nothing left to start: retire the dead slots
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
             i += (int64_t)gridDim.x * blockDim.x)
            P.flags[checked_slot(src_at(src, i), P, ctl)] = PF_RETIRED;
        return;
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int added = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < count; base += stride) {
        const int64_t i = base + threadIdx.x;
        int64_t slot = -1;
        bool want = false;
        if (i < count) {
            if (queued || fq) {
                slot = checked_slot(src_at(src, i), P, ctl);
                want = true;
            } else {
                slot = i;
                want = (P.flags[slot] & (PF_ALIVE | PF_RETIRED)) == 0;
            }
        }
        const unsigned b = __ballot_sync(FULL, want);
        if (b == 0u) continue;
        const int leader = __ffs(b) - 1;
        unsigned long long wbase = 0ull;
        if (lane_id() == leader) wbase = atomicAdd(&ctl->next, (unsigned long long)__popc(b));
        wbase = __shfl_sync(FULL, wbase, leader);
        bool got = false;
        if (want) {
            const long long wk = (long long)(wbase + __popc(b & lanes_below()));
            if (wk < total) {
                const int p = problem_of_work(work_off, n_prob, wk);
                const ProblemDev& pd = probs[p];
                init_particle<EIG>(P, slot, pd, p, pd.first + (wk - work_off[p]), c.derivatives ? pd.M : 0);
                got = true;
            } else {
                P.flags[slot] = PF_RETIRED;
            }
        }
        if (queued) {
            int pos = warp_append(&ctl->n_xs[par], got);
            if (got) queue_put(P.q_xs[par], pos, slot, P, ctl);
            pos = warp_append(&ctl->n_adv[par], got);
            if (got) queue_put(P.q_adv[par], pos, slot, P, ctl);
        } else if (fq) {
            ring_push(P, ctl, RQ_XS, got, slot);
        }
        const unsigned gm = __ballot_sync(FULL, got);
        if (lane_id() == 0) added += __popc(gm);
    }
    if (lane_id() == 0 && added) atomicAdd(&ctl->n_alive, added);
}

// The transport lookup of the particle in `slot` if it needs one: Sigma_t,
// Sigma_a (nuSigma_f) and the running sums C_i; returns whether it did.
template <typename T, bool EIG>
__device__ __forceinline__ bool lookup_slot(const Tables& t, const Particles& P, int64_t slot)
{
    const uint8_t f = P.flags[slot];
    if (!(f & PF_NEED_XS)) return false;
    double st, sa;
#if MCX_TRANSPORT_PAIRS
    float2* cum2 = reinterpret_cast<float2*>(P.cum + slot * P.cum_stride);
    if (EIG) {
        double nf;
        macro_transport_pair<true>(t, P.mat[slot], P.E[slot], st, sa, cum2, &nf);
        P.sig_nf[slot] = nf;
    } else {
        macro_transport_pair<false>(t, P.mat[slot], P.E[slot], st, sa, cum2);
    }
#else
    if (EIG) {
        double nf;
        macro_transport<T, true>(t, P.mat[slot], P.E[slot], st, sa, P.cum + slot * P.cum_stride, &nf);
        P.sig_nf[slot] = nf;
    } else {
        macro_transport<T>(t, P.mat[slot], P.E[slot], st, sa, P.cum + slot * P.cum_stride);
    }
#endif
    P.sig_ta[slot] = make_double2(st, sa);
    P.flags[slot] = f & (uint8_t)~PF_NEED_XS;
    return true;
}

template <typename T, bool EIG>
__global__ void __launch_bounds__(1024) k_lookup(LoopConfig c, Tables t, Particles P, RunCtl* ctl)
{
    if (ctl->error) return;
    const bool fq = c.mode == MCX_QUEUED_FULLEST;
    if (fq && ctl->sel != SEL_XS) return;
    const int par = ctl->parity;
    Src src = all_slots(P);
    if (c.mode == MCX_QUEUED)
        src = ctl->sorted ? plain_list(P.q_sorted, ctl->n_xs[par]) : plain_list(P.q_xs[par], ctl->n_xs[par]);
    else if (fq)
        src = ctl->sorted ? plain_list(P.q_sorted, (int64_t)(ctl->sel_end - ctl->sel_begin))
                          : ring_segment(P, ctl);
    const int adv = RQ_ADV0 + ctl->adv_recv;
    const int64_t count = src.n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
#if MCX_TRANSPORT_WARP_TAIL
    // Few lookups (the tail of the loop): one warp per particle, all of them
    // in one round of the grid; the same values as the per-thread path.
    if (count * 32 <= stride) {
        const int lane = lane_id();
        const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        if (w < count) {   // the whole warp
            const int64_t slot = checked_slot(src_at(src, w), P, ctl);
            const uint8_t f = P.flags[slot];
            const bool act = (f & PF_NEED_XS) != 0;
            if (act) {
                double st, sa, nf = 0.0;
#if MCX_TRANSPORT_PAIRS
                macro_transport_pair_warp<EIG>(t, P.mat[slot], P.E[slot], st, sa,
                                               reinterpret_cast<float2*>(P.cum + slot * P.cum_stride), &nf);
#else
                macro_transport_warp<T, EIG>(t, P.mat[slot], P.E[slot], st, sa, P.cum + slot * P.cum_stride,
                                             &nf);
#endif
                if (lane == 0) {
                    if (EIG) P.sig_nf[slot] = nf;
                    P.sig_ta[slot] = make_double2(st, sa);
                    P.flags[slot] = f & (uint8_t)~PF_NEED_XS;
                }
            }
            if (fq) ring_push(P, ctl, adv, act && lane == 0, slot);
        }
        return;
    }
#endif
#if MCX_LOOKUP_CLAIM
    if (c.mode == MCX_QUEUED) {
        // Warps claim 32-entry chunks of the (binned) queue front to back:
        // the lookups in flight at any time sit in a narrow slice of
        // (material, energy), and no warp idles while another still holds a
        // grid-stride share.
        const int lane = lane_id();
        for (;;) {
            unsigned long long b0 = 0ull;
            if (lane == 0) b0 = atomicAdd(&ctl->lk_claim, 32ull);
            const int64_t b = (int64_t)__shfl_sync(FULL, b0, 0);
            if (b >= count) break;
            const int64_t i = b + lane;
            if (i < count) lookup_slot<T, EIG>(t, P, checked_slot(src_at(src, i), P, ctl));
        }
        return;
    }
#endif
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < count; base += stride) {
        const int64_t i = base + threadIdx.x;
        int64_t slot = -1;
        bool act = false;
        if (i < count) {
            slot = checked_slot(src_at(src, i), P, ctl);
            act = lookup_slot<T, EIG>(t, P, slot);
        }
        if (fq) ring_push(P, ctl, adv, act, slot);
    }
}

template <bool EIG>
__global__ void __launch_bounds__(1024) k_advance(LoopConfig c, Particles P, const ProblemDev* probs,
                                                  RunCtl* ctl)
{
    if (ctl->error) return;
    const bool queued = c.mode == MCX_QUEUED;
    const bool fq = c.mode == MCX_QUEUED_FULLEST;
    if (fq && ctl->sel != SEL_ADV) return;
    const int par = ctl->parity;
    Src src = all_slots(P);
    // Queued mode: the list holds every live particle (each flies once per
    // iteration); when it covers at least three quarters of the slots the
    // flight scans the slots instead (coalesced state loads, not the order
    // the previous kernels wrote the list in); the tail of the loop, and the
    // emptying slots of an eigenvalue generation, read the list
    // (1.402e7 -> 1.467e7 particles/s against always scanning; eigenvalue
    // 5.03e6 -> 6.04e6).
    if (queued && (int64_t)ctl->n_adv[par] * 4 < P.cap * 3) src = plain_list(P.q_adv[par], ctl->n_adv[par]);
    else if (fq) src = ring_segment(P, ctl);
    const int adv = RQ_ADV0 + ctl->adv_recv;   // the ring not being read
    const int64_t count = src.n;
    const int M = c.derivatives;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < count; base += stride) {
        const int64_t i = base + threadIdx.x;
        int64_t slot = -1;
        bool act = false;
        if (i < count) {
            slot = checked_slot(src_at(src, i), P, ctl);
            act = src.list ? true : (P.flags[slot] & PF_ALIVE) != 0;
        }
        bool scored = false, dies = false, coll = false, survive = false, need_xs = false;
        int outcome = -1;
        int32_t pidx = 0;
        double d = 0.0, xabs = 0.0;
        double* tal_flux = nullptr;
        double* tal_abs = nullptr;
        int64_t tal_i = 0;
        double k_tl = 0.0;
        double Wl[MCX_MAX_DMAT] = {0.0, 0.0, 0.0, 0.0};
        int32_t m = 0;
        if (act) {
            pidx = P.prob[slot];
            const ProblemDev& pd = probs[pidx];
            State q = load_state(P, slot, pd.lattice_n);
            const int64_t h = P.hist[slot];
            uint32_t n = P.rng_n[slot];
            const double xi = uniform_at(pd.key, h, n);
            n += 1;
            const double2 ta = P.sig_ta[slot];
            const double sig_t = ta.x, sig_a = ta.y;
            m = P.mat[slot];
            int surf;
#if MCX_TRANSPORT_ONE_DIV
            // collide iff the surface's t = num / den exceeds L / Sigma_t
            // (num Sigma_t > L den, den > 0): one division, for the distance taken
            const double L = neg_log_uniform(xi);
            double sn, sd;
            surface_candidate(pd, q, surf, sn, sd);
            bool collide;
            if (!(sig_t > 0.0)) collide = false;
            else if (!ne0(sd)) collide = true;
            else collide = !(sn * sig_t <= L * sd);
#if MCX_TRANSPORT_CONVERGED
            // one division for the whole warp, collisions and crossings alike
            if (!collide && !ne0(sd)) {
                d = INF;
            } else {
                d = (collide ? L : sn) / (collide ? sig_t : sd);
                if (lt0(d)) d = 0.0;   // a collision's L / Sigma_t is positive
            }
#else
            if (collide) {
                d = L / sig_t;
            } else if (sd == 0.0) {
                d = INF;
            } else {
                d = sn / sd;
                if (d < 0.0) d = 0.0;
            }
#endif
#else
            const double dcol = sig_t > 0.0 ? -log(xi) / sig_t : INF;
            const double dsurf = surface_distance(pd, q, surf);
            const bool collide = !(dsurf <= dcol);
            d = collide ? dcol : dsurf;
#endif
            uint8_t fl = P.flags[slot];
            if (isinf(d)) {
                dies = true;
                outcome = OUT_LEAK_OTHER;
            } else {
#if MCX_TRANSPORT_GEOM_FMA
                q.x = fma(d, q.u, q.x);
                q.y = fma(d, q.v, q.y);
                q.z = fma(d, q.w, q.z);
#else
                q.x = q.x + d * q.u;
                q.y = q.y + d * q.v;
                q.z = q.z + d * q.w;
#endif
                int32_t bin;
                if (pd.geometry == MCX_GEOM_INFINITE)
                    bin = (int32_t)bsearch_window(pd.ebin_edges, 0, pd.n_ebins - 1, ebits(P.E[slot]));
                else
                    bin = region_of(pd, q);
                const int64_t b = batch_of(pd, h);
                tal_i = b * pd.nb + bin;
                tal_flux = pd.flux + tal_i;
                tal_abs = pd.absorb + tal_i;
                scored = true;
#if MCX_BOUNDS_CHECK
                if (!MCX_IN_BOUNDS(tal_i >= 0 && tal_i < (int64_t)pd.n_batches * pd.nb, BC_TALLY, tal_i)) {
                    atomicCAS(&ctl->error, 0, MCX_ERR_BOUNDS);
                    scored = false;
                }
#endif
                xabs = d * sig_a;
                if (EIG) k_tl = d * P.sig_nf[slot];
                if (M > 0) {
                    for (int mm = 0; mm < M; ++mm) Wl[mm] = P.W[(int64_t)mm * P.stride + slot];
                    for (int mm = 0; mm < M; ++mm) {
                        if (mm == m) {
                            Wl[mm] = Wl[mm] - sig_t * d;
                            if (collide) Wl[mm] = Wl[mm] + 1.0;
                        }
                    }
                    for (int mm = 0; mm < M; ++mm) P.W[(int64_t)mm * P.stride + slot] = Wl[mm];
                }
                if (!collide) {
                    const int o = cross_surface(pd, q, surf);
                    if (o >= 0) {
                        dies = true;
                        outcome = o;
                    } else {
                        survive = true;
                        const int32_t nm = __ldg(pd.region_material + region_of(pd, q));
                        if (nm != m) {
                            need_xs = true;
                            P.mat[slot] = nm;
                        }
                        fl = (uint8_t)((fl & ~(PF_INPIN | PF_NEED_XS)) | (q.inpin ? PF_INPIN : 0) |
                                       (need_xs ? PF_NEED_XS : 0));
                        P.cell[slot] = q.ci * (pd.lattice_n > 0 ? pd.lattice_n : 1) + q.cj;
                        P.w[slot] = q.w;
                    }
                } else {
                    coll = true;
                    fl |= PF_COLLIDE;
                }
                P.x[slot] = q.x;
                P.y[slot] = q.y;
                P.z[slot] = q.z;
            }
            P.rng_n[slot] = n;
            P.flags[slot] = fl;
        }
        if (EIG) warp_add(&probs[0].eig->k_tl, k_tl, scored);
        // ---- warp-first tally reduction
        const unsigned sm = __ballot_sync(FULL, scored);
#if MCX_TALLY_TREE
        if (sm) {
            // unscored lanes share the key 0, a group whose sums are not added
            const unsigned grp = __match_any_sync(FULL, scored ? (unsigned long long)tal_flux : 0ull);
            const bool lead = scored && lane_id() == __ffs(grp) - 1;
            double v[2] = {scored ? d : 0.0, scored ? xabs : 0.0};
            group_sum(grp, v);
            if (lead) {
                atomicAdd(tal_flux, v[0]);
                atomicAdd(tal_abs, v[1]);
            }
            for (int mm = 0; mm < M; ++mm) {
                double w[2] = {scored ? d * Wl[mm] : 0.0,
                               scored ? xabs * Wl[mm] + (mm == m ? xabs : 0.0) : 0.0};
                group_sum(grp, w);
                if (lead) {
                    const ProblemDev& pd = probs[pidx];
                    atomicAdd(pd.dflux + tal_i * M + mm, w[0]);
                    atomicAdd(pd.dabsorb + tal_i * M + mm, w[1]);
                }
            }
        }
#else
        if (scored) {
            const unsigned grp = __match_any_sync(sm, (unsigned long long)tal_flux);
            const int leader = __ffs(grp) - 1;
            double sf = 0.0, sa = 0.0;
            for (unsigned g = grp; g; g &= g - 1u) {
                const int src = __ffs(g) - 1;
                sf += __shfl_sync(grp, d, src);
                sa += __shfl_sync(grp, xabs, src);
            }
            if (lane_id() == leader) {
                atomicAdd(tal_flux, sf);
                atomicAdd(tal_abs, sa);
            }
            if (M > 0) {
                const ProblemDev& pd = probs[pidx];
                for (int mm = 0; mm < M; ++mm) {
                    const double vf = d * Wl[mm];
                    const double va = xabs * Wl[mm] + (mm == m ? xabs : 0.0);
                    double s1 = 0.0, s2 = 0.0;
                    for (unsigned g = grp; g; g &= g - 1u) {
                        const int src = __ffs(g) - 1;
                        s1 += __shfl_sync(grp, vf, src);
                        s2 += __shfl_sync(grp, va, src);
                    }
                    if (lane_id() == leader) {
                        atomicAdd(pd.dflux + tal_i * M + mm, s1);
                        atomicAdd(pd.dabsorb + tal_i * M + mm, s2);
                    }
                }
            }
        }
#endif
        finish_deaths<EIG>(dies, outcome, slot, pidx, probs, P, ctl, M, c.mode, par);
        if (queued) {
            int pos = warp_append(&ctl->n_coll, coll);
            if (coll) queue_put(P.q_coll, pos, slot, P, ctl);
            pos = warp_append(&ctl->n_adv[par ^ 1], survive);
            if (survive) queue_put(P.q_adv[par ^ 1], pos, slot, P, ctl);
            pos = warp_append(&ctl->n_xs[par ^ 1], need_xs);
            if (need_xs) queue_put(P.q_xs[par ^ 1], pos, slot, P, ctl);
        } else if (fq) {
            ring_push(P, ctl, RQ_COLL, coll, slot);
            ring_push(P, ctl, RQ_XS, survive && need_xs, slot);
            ring_push(P, ctl, adv, survive && !need_xs, slot);
        }
    }
}

// Collision: species j = the first with xi1 * Sigma_t < C_j (C_j the running
// sum of N_i (sigma_s,i + sigma_a,i) in stored order; the last species if
// none); absorption if xi2 * sigma_t,j < sigma_a,j (analog); otherwise
// elastic scattering isotropic in the centre-of-mass frame, killed below
// E_cut.
template <typename T, bool EIG>
__global__ void __launch_bounds__(1024) k_collide(LoopConfig c, Tables t, Particles P,
                                                  const ProblemDev* probs, RunCtl* ctl)
{
    if (ctl->error) return;
    const bool queued = c.mode == MCX_QUEUED;
    const bool fq = c.mode == MCX_QUEUED_FULLEST;
    if (fq && ctl->sel != SEL_COLL) return;
    const int par = ctl->parity;
    Src src = all_slots(P);
    if (queued)
        src = plain_list(P.q_coll, ctl->n_coll);
    else if (fq)
        src = ctl->sorted ? plain_list(P.q_sorted, (int64_t)(ctl->sel_end - ctl->sel_begin))
                          : ring_segment(P, ctl);
    const int64_t count = src.n;
    const int M = c.derivatives;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < count; base += stride) {
        const int64_t i = base + threadIdx.x;
        int64_t slot = -1;
        bool act = false;
        if (i < count) {
            slot = checked_slot(src_at(src, i), P, ctl);
            act = src.list ? true : (P.flags[slot] & PF_COLLIDE) != 0;
        }
        bool dies = false, survive = false;
        int outcome = -1;
        int32_t pidx = 0;
        double* tal_coll = nullptr;
        int64_t tal_i = 0;
        double k_col = 0.0;
        int64_t n_new = 0;
        uint32_t seq0 = 0u;
        FissionSite site;
        if (act) {
            pidx = P.prob[slot];
            const ProblemDev& pd = probs[pidx];
            const int64_t h = P.hist[slot];
            uint32_t n = P.rng_n[slot];
            P.ncoll[slot] += 1u;
            tal_i = batch_of(pd, h) * N_OUT + OUT_COLLISIONS;
            tal_coll = pd.outcome + tal_i;
            const double xi1 = uniform_at(pd.key, h, n);
            const double xi2 = uniform_at(pd.key, h, n + 1);
            const double mu = uniform_signed(pd.key, h, n + 2);   // 2 xi3 - 1
            n += 3;
            if (EIG) {
                // fission sites of this collision, banked before the reaction
                // is decided: floor(nuSigma_f / Sigma_t / k_norm + xi4)
                const double xi4 = uniform_at(pd.key, h, n);
                n += 1;
                const double yield = P.sig_nf[slot] / P.sig_ta[slot].x;
                k_col = yield;
                const double fl = floor(yield / pd.k_norm + xi4);
                const double lim = (double)pd.bank_cap + 1.0;   // overflow is reported, not looped on
                n_new = fl > 0.0 ? (int64_t)(fl < lim ? fl : lim) : 0;
                site.x = P.x[slot];
                site.y = P.y[slot];
                site.z = P.z[slot];
                site.cell = P.cell[slot];
                site.inpin = (P.flags[slot] & PF_INPIN) ? 1 : 0;
                seq0 = P.nsite[slot];
                P.nsite[slot] = seq0 + (uint32_t)n_new;
            }
            const double E = P.E[slot];
            int32_t m = P.mat[slot];
#if MCX_BOUNDS_CHECK
            if (!MCX_IN_BOUNDS(m >= 0 && m < t.n_materials, BC_SPECIES, m)) {
                atomicCAS(&ctl->error, 0, MCX_ERR_BOUNDS);
                m = 0;
            }
#endif
            const double target = xi1 * P.sig_ta[slot].x;
            const int64_t eb = search_key(E);
            const int32_t hb = t.H > 0 ? hash_bin(t, E, eb) : 0;
            // species choice: the first i with target < C_i, C_i the running
            // sums the lookup kernel stored for this energy and material (the
            // same FP64 values a sequential pass would form); the last species
            // if none.  C is non-decreasing and non-negative, so a binary
            // search on the bit patterns finds the first C_i > target.
            const int32_t i0 = __ldg(t.moff + m), n_sp = __ldg(t.moff + m + 1) - i0;
            int32_t lo = 0, hi = n_sp - 1;
#if MCX_TRANSPORT_PAIRS
            // C_i are normalised FP32 pairs, so their order is the order of
            // (hi, lo); the target is compared as a pair too
            const float2* cum2 = reinterpret_cast<const float2*>(P.cum + slot * P.cum_stride);
            const float2 tp = energy_pair(target);
            while (lo < hi) {
                const int32_t mid = (lo + hi) >> 1;
                const float2 cm = cum2[mid];
                if (tp.x < cm.x || (tp.x == cm.x && tp.y < cm.y)) hi = mid;
                else lo = mid + 1;
            }
#else
            const double* cum = P.cum + slot * P.cum_stride;
            const int64_t tb = ebits(target);
            while (lo < hi) {
                const int32_t mid = (lo + hi) >> 1;
                if (tb < ebits(cum[mid])) hi = mid;
                else lo = mid + 1;
            }
#endif
            const int32_t j = __ldg(t.msp + i0 + lo);
            double st_j, sa_j;
            {
                const int64_t k = species_index(t, j, eb, hb);
                const int64_t g0 = __ldg(t.goff + j);
                const int64_t last = __ldg(t.goff + j + 1) - 2;
                double unused = 0.0;
                species_transport<T, false>(t, E, g0 + k, last, st_j, sa_j, unused);
            }
            uint8_t fl = (uint8_t)(P.flags[slot] & ~PF_COLLIDE);
            if (xi2 * st_j < sa_j) {
                dies = true;
                outcome = OUT_ABSORBED;
            } else {
                const double A = __ldg(t.awr + j);
                const double num = A * A + 2.0 * A * mu + 1.0;
#if MCX_TRANSPORT_KINEMATICS
                const double E_new = (E * num) * __ldg(t.inv_a1sq + j);   // (A + 1)^-2 stored per species
#else
                const double den = (A + 1.0) * (A + 1.0);
                const double E_new = E * (num / den);
#endif
                if (E_new < pd.E_cut) {
                    dies = true;
                    outcome = OUT_CUTOFF;
                } else {
#if MCX_TRANSPORT_RECIP_DIR
                    double mu_lab = (1.0 + A * mu) * rsqrt(num);
#else
                    double mu_lab = (1.0 + A * mu) / sqrt(num);
#endif
                    if (mu_lab > 1.0) mu_lab = 1.0;
                    if (mu_lab < -1.0) mu_lab = -1.0;
                    double u = P.u[slot], v = P.v[slot], w = P.w[slot];
#if MCX_TRANSPORT_KINEMATICS
                    double cr, sr, rho;
                    azimuth_raw(pd.key, h, n, cr, sr, rho);
                    rotate_raw(u, v, w, mu_lab, cr, sr, rho);
#else
                    double cphi, sphi;
                    azimuth(pd.key, h, n, cphi, sphi);
                    rotate(u, v, w, mu_lab, cphi, sphi);
#endif
                    P.u[slot] = u;
                    P.v[slot] = v;
                    P.w[slot] = w;
                    P.E[slot] = E_new;
                    fl |= PF_NEED_XS;
                    survive = true;
                }
            }
            P.rng_n[slot] = n;
            P.flags[slot] = fl;
        }
        if (EIG) {
            const ProblemDev& p0 = probs[0];
            warp_add(&p0.eig->k_col, k_col, act);
            const int64_t hrel = act ? P.hist[slot] - p0.first : 0;
            for (int64_t s = 0;; ++s) {
                const bool want = act && s < n_new;
                const unsigned b = __ballot_sync(FULL, want);
                if (b == 0u) break;
                const int leader = __ffs(b) - 1;
                unsigned long long base = 0ull;
                if (lane_id() == leader) base = atomicAdd(&p0.eig->banked, (unsigned long long)__popc(b));
                base = __shfl_sync(FULL, base, leader);
                if (want) {
                    const unsigned long long pos = base + __popc(b & lanes_below());
                    if (pos < (unsigned long long)p0.bank_cap) {
                        p0.bank[pos] = site;
                        p0.bank_key[pos] = make_int2((int32_t)hrel, (int32_t)(seq0 + (uint32_t)s));
                    }
                }
            }
        }
        // collision-count tally (+ derivative), warp-first
        const unsigned am = __ballot_sync(FULL, act);
        if (am) {
            const unsigned grp = __match_any_sync(FULL, act ? (unsigned long long)tal_coll : 0ull);
            const bool lead = act && lane_id() == __ffs(grp) - 1;
            if (lead) atomicAdd(tal_coll, (double)__popc(grp));
            for (int mm = 0; mm < M; ++mm) {
                double wv[1] = {act ? P.W[(int64_t)mm * P.stride + slot] : 0.0};
                group_sum(grp, wv);
                if (lead) atomicAdd(probs[pidx].doutcome + tal_i * M + mm, wv[0]);
            }
        }
        finish_deaths<EIG>(dies, outcome, slot, pidx, probs, P, ctl, M, c.mode, par);
        if (queued) {
            int pos = warp_append(&ctl->n_xs[par ^ 1], survive);
            if (survive) queue_put(P.q_xs[par ^ 1], pos, slot, P, ctl);
            pos = warp_append(&ctl->n_adv[par ^ 1], survive);
            if (survive) queue_put(P.q_adv[par ^ 1], pos, slot, P, ctl);
        } else if (fq) {
            ring_push(P, ctl, RQ_XS, survive, slot);
        }
    }
}

__global__ void k_bookkeep(RunCtl* ctl)
{
    const int p = ctl->parity;
    ctl->ev_count[0] += ctl->n_xs[p];
    ctl->ev_count[1] += ctl->n_adv[p];
    ctl->ev_count[2] += ctl->n_coll;
    ctl->n_xs[p] = 0;
    ctl->n_adv[p] = 0;
    ctl->n_dead[p] = 0;
    ctl->n_coll = 0;
    ctl->parity = p ^ 1;
    ctl->sorted = 0;
    ctl->lk_claim = 0ull;
    if (!ctl->done) {
        ctl->iters += 1;
        if (ctl->n_alive == 0 && (long long)ctl->next >= ctl->total) {
            ctl->done = 1;
        } else if (ctl->iters >= ctl->max_iters) {
            ctl->error = MCX_ERR_ITER_LIMIT;
            ctl->done = 1;
        }
    }
}

// Kernel timing runs (queued mode): the running-sum row lengths this
// iteration's lookups will write, each material's species count rounded up
// to a multiple of 4 (the rows are stored four entries at a time).
__global__ void k_census(Particles P, const int32_t* __restrict__ moff, RunCtl* ctl)
{
    const int par = ctl->parity;
    const int64_t n = ctl->n_xs[par];
    long long s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t m = P.mat[checked_slot(P.q_xs[par][i], P, ctl)];
        s += ((long long)(__ldg(moff + m + 1) - __ldg(moff + m)) + 3) & ~3LL;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd((unsigned long long*)&ctl->ev_count[3], (unsigned long long)s);
}

// Fullest-queue mode: retire the free-slot ring the refill just drained, stop
// when no particle is left in any queue, and hand the fullest of the lookup,
// flight and collision queues to this step's event kernel (ties go to the
// earlier event of the sequence lookup, flight, collision).  One thread.
__global__ void k_fq_select(RunCtl* ctl, long long cap)
{
    ctl->sel = -1;
    ctl->sorted = 0;
    if (ctl->error || ctl->done) return;
    ctl->rq_head[RQ_DEAD] = ctl->rq_tail[RQ_DEAD];
    const int adv = RQ_ADV0 + ctl->adv_recv;
    const unsigned long long nx = ctl->rq_tail[RQ_XS] - ctl->rq_head[RQ_XS];
    const unsigned long long na = ctl->rq_tail[adv] - ctl->rq_head[adv];
    const unsigned long long nc = ctl->rq_tail[RQ_COLL] - ctl->rq_head[RQ_COLL];
    const unsigned long long idle = ctl->rq_tail[adv ^ 3] - ctl->rq_head[adv ^ 3];
    if (nx > (unsigned long long)cap || na > (unsigned long long)cap || nc > (unsigned long long)cap ||
        idle != 0ull) {
        ctl->error = MCX_ERR_STATE;   // a queue invariant broke: stop before any wrapped read
        ctl->done = 1;
        return;
    }
    if (nx == 0ull && na == 0ull && nc == 0ull) {
        ctl->done = 1;
        return;
    }
    if (ctl->iters >= ctl->max_iters) {
        ctl->error = MCX_ERR_ITER_LIMIT;
        ctl->done = 1;
        return;
    }
    ctl->iters += 1;
    int sel = SEL_XS, ring = RQ_XS;
    unsigned long long n = nx;
    if (na > n) {
        sel = SEL_ADV;
        ring = adv;
        n = na;
    }
    if (nc > n) {
        sel = SEL_COLL;
        ring = RQ_COLL;
    }
    ctl->sel = sel;
    ctl->sel_count[sel] += 1;
    ctl->sel_ring = ring;
    ctl->sel_begin = ctl->rq_head[ring];
    ctl->sel_end = ctl->rq_tail[ring];
    ctl->rq_head[ring] = ctl->rq_tail[ring];
    if (sel == SEL_ADV) ctl->adv_recv ^= 1;
}

// ---- binning of a queue by (material, log-energy bucket)
__device__ __forceinline__ int sort_key(const LoopConfig& c, double E, int32_t m)
{
    float fb = (logf((float)E) - c.sort_ln_lo) * c.sort_scale;
    int b = fb >= 0.f ? (int)fb : 0;
    if (b >= c.n_ebuckets) b = c.n_ebuckets - 1;
    return m * c.n_ebuckets + b;
}

// which: 0 = XS queue (consumed side), 1 = collision queue, 2 = the segment
// the fullest-queue select kernel chose, when it is a lookup or collision one
__device__ __forceinline__ Src sort_source(const Particles& P, const RunCtl* ctl, int which)
{
    const int par = ctl->parity;
    if (which == 2) return ring_segment(P, ctl);
    return which == 0 ? plain_list(P.q_xs[par], ctl->n_xs[par]) : plain_list(P.q_coll, ctl->n_coll);
}

__global__ void k_sort_decide(LoopConfig c, RunCtl* ctl, int which)
{
    const int par = ctl->parity;
    long long n = which == 0 ? ctl->n_xs[par] : ctl->n_coll;
    if (which == 2)
        n = (ctl->sel == SEL_XS || ctl->sel == SEL_COLL) ? (long long)(ctl->sel_end - ctl->sel_begin) : 0;
    ctl->sorted = (!ctl->error && c.sort_period > 0 && (ctl->iters % c.sort_period) == 0 &&
                   n >= c.sort_threshold && n > 0)
                      ? 1
                      : 0;
}

__global__ void k_sort_count(LoopConfig c, Particles P, RunCtl* ctl, int which)
{
    extern __shared__ uint32_t hist[];
    if (!ctl->sorted) return;
    const Src src = sort_source(P, ctl, which);
    const int64_t n = src.n;
    for (int i = threadIdx.x; i < c.n_sort_bins; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = (int32_t)checked_slot(src_at(src, i), P, ctl);
        atomicAdd(&hist[sort_key(c, P.E[s], P.mat[s])], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < c.n_sort_bins; i += blockDim.x)
        if (hist[i]) atomicAdd(&P.bins[i], hist[i]);
}

// Exclusive scan of the bin counts (one block).
__global__ void k_sort_scan(LoopConfig c, Particles P, RunCtl* ctl)
{
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry;
    if (!ctl->sorted) return;
    if (threadIdx.x == 0) carry = 0u;
    __syncthreads();
    const int nb = c.n_sort_bins;
    for (int base = 0; base < nb; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < nb ? P.bins[i] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, x, o);
            if (lane_id() >= o) x += y;
        }
        if (lane_id() == 31) warp_sums[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            const int nw = blockDim.x >> 5;
            uint32_t s = threadIdx.x < nw ? warp_sums[threadIdx.x] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL, s, o);
                if (lane_id() >= o) s += y;
            }
            if (threadIdx.x < nw) warp_sums[threadIdx.x] = s;
        }
        __syncthreads();
        const uint32_t before = (threadIdx.x >> 5) ? warp_sums[(threadIdx.x >> 5) - 1] : 0u;
        if (i < nb) P.bins[i] = carry + before + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += before + x;
        __syncthreads();
    }
}

// Scatter into the binned list.  Each round a block takes blockDim.x *
// kSortPer entries; their ranks within the round come from a shared-memory
// histogram, and one global atomic per non-empty bin reserves the round's
// range of that bin (instead of one per distinct key per warp, all
// contending on the same few hundred counters).  The order inside a bin is
// free: no result depends on it.
constexpr int kSortPer = 8;
__global__ void k_sort_scatter(LoopConfig c, Particles P, RunCtl* ctl, int which)
{
    extern __shared__ uint32_t sh[];
    if (!ctl->sorted) return;
    const Src src = sort_source(P, ctl, which);
    const int64_t n = src.n;
    const int nb = c.n_sort_bins;
    const int64_t tile = (int64_t)blockDim.x * kSortPer;
    for (int64_t base = (int64_t)blockIdx.x * tile; base < n; base += (int64_t)gridDim.x * tile) {
        for (int b = threadIdx.x; b < nb; b += blockDim.x) sh[b] = 0u;
        __syncthreads();
        int32_t sl[kSortPer];
        int key[kSortPer];
        uint32_t rank[kSortPer];
#pragma unroll
        for (int r = 0; r < kSortPer; ++r) {
            const int64_t i = base + (int64_t)r * blockDim.x + threadIdx.x;
            key[r] = -1;
            sl[r] = 0;
            rank[r] = 0u;
            if (i < n) {
                sl[r] = (int32_t)checked_slot(src_at(src, i), P, ctl);
                key[r] = sort_key(c, P.E[sl[r]], P.mat[sl[r]]);
                rank[r] = atomicAdd(&sh[key[r]], 1u);
            }
        }
        __syncthreads();
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const uint32_t cnt = sh[b];
            if (cnt) sh[b] = atomicAdd(&P.bins[b], cnt);
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kSortPer; ++r)
            if (key[r] >= 0) queue_put(P.q_sorted, sh[key[r]] + rank[r], sl[r], P, ctl);
        __syncthreads();
    }
}

}  // namespace

int launch_run_init(const LoopConfig& c, const Particles& P, RunCtl* ctl, long long total,
                    int n_prob, long long max_iters, cudaStream_t st)
{
    k_init_nlog<<<1, 256, 0, st>>>();   // the flight-length table (same values every time)
    k_run_init<<<c.grid, 256, 0, st>>>(P, ctl, total, n_prob, max_iters, c.mode);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

static int launch_sort(const LoopConfig& c, const Particles& P, RunCtl* ctl, int which,
                       cudaStream_t st)
{
    if (cudaMemsetAsync(P.bins, 0, sizeof(uint32_t) * (size_t)(c.n_sort_bins + 1), st) != cudaSuccess)
        return -1;
    k_sort_decide<<<1, 1, 0, st>>>(c, ctl, which);
    k_sort_count<<<c.grid, c.block, sizeof(uint32_t) * c.n_sort_bins, st>>>(c, P, ctl, which);
    k_sort_scan<<<1, 1024, 0, st>>>(c, P, ctl);
    k_sort_scatter<<<c.grid, c.block, sizeof(uint32_t) * c.n_sort_bins, st>>>(c, P, ctl, which);
    return 4;
}

template <bool EIG>
static int launch_iteration_t(const LoopConfig& c, const Tables& t, const Particles& P,
                              const ProblemDev* probs, const int64_t* work_off, RunCtl* ctl,
                              cudaStream_t st, const cudaEvent_t* ev)
{
    int k = 0;
    const bool sorting = c.mode != MCX_QUEUELESS && c.sort_period > 0 && c.n_sort_bins > 0;
    const bool f32 = t.precision == MCX_FP32;
    k_refill<EIG><<<c.grid, c.block, 0, st>>>(c, P, probs, work_off, ctl);
    ++k;
    if (c.mode == MCX_QUEUED_FULLEST) {
        // one step: the event kernels not selected return at once
        k_fq_select<<<1, 1, 0, st>>>(ctl, (long long)P.cap);
        ++k;
        if (sorting) k += launch_sort(c, P, ctl, 2, st);
        if (ev) cudaEventRecord(ev[0], st);
        if (f32) k_lookup<float, EIG><<<c.grid, c.block, 0, st>>>(c, t, P, ctl);
        else k_lookup<double, EIG><<<c.grid, c.block, 0, st>>>(c, t, P, ctl);
        if (ev) cudaEventRecord(ev[1], st);
        k_advance<EIG><<<c.grid, c.block, 0, st>>>(c, P, probs, ctl);
        if (ev) cudaEventRecord(ev[2], st);
        if (f32) k_collide<float, EIG><<<c.grid, c.block, 0, st>>>(c, t, P, probs, ctl);
        else k_collide<double, EIG><<<c.grid, c.block, 0, st>>>(c, t, P, probs, ctl);
        if (ev) cudaEventRecord(ev[3], st);
        k += 3;
        if (cudaGetLastError() != cudaSuccess) return -1;
        return k;
    }
    if (sorting) k += launch_sort(c, P, ctl, 0, st);
    if (ev) {
        if (c.mode == MCX_QUEUED) k_census<<<c.grid, 256, 0, st>>>(P, t.moff, ctl);
        cudaEventRecord(ev[0], st);
    }
    if (f32) k_lookup<float, EIG><<<c.grid, c.block, 0, st>>>(c, t, P, ctl);
    else k_lookup<double, EIG><<<c.grid, c.block, 0, st>>>(c, t, P, ctl);
    ++k;
    if (ev) cudaEventRecord(ev[1], st);
    k_advance<EIG><<<c.grid, c.block, 0, st>>>(c, P, probs, ctl);
    ++k;
    if (ev) cudaEventRecord(ev[2], st);
    // (the collision queue is not binned: one species per collision gains
    // less from the locality than the binning costs -- 654 -> 640 ms per 1e7
    // lattice histories without it)
    if (f32) k_collide<float, EIG><<<c.grid, c.block, 0, st>>>(c, t, P, probs, ctl);
    else k_collide<double, EIG><<<c.grid, c.block, 0, st>>>(c, t, P, probs, ctl);
    ++k;
    if (ev) cudaEventRecord(ev[3], st);
    k_bookkeep<<<1, 1, 0, st>>>(ctl);
    ++k;
    if (cudaGetLastError() != cudaSuccess) return -1;
    return k;
}

// Kernels of one iteration; eigenvalue generations use the instantiations
// that bank fission sites, fixed-source runs the ones without that code.
int launch_iteration(const LoopConfig& c, const Tables& t, const Particles& P,
                     const ProblemDev* probs, const int64_t* work_off, RunCtl* ctl,
                     cudaStream_t st, const cudaEvent_t* ev)
{
    return c.eigen ? launch_iteration_t<true>(c, t, P, probs, work_off, ctl, st, ev)
                   : launch_iteration_t<false>(c, t, P, probs, work_off, ctl, st, ev);
}

// Philox uniforms of one history stream (test hook).
__global__ void k_debug_uniforms(uint2 key, uint64_t hist, uint32_t first, int64_t n, double* out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = uniform_at(key, hist, first + (uint32_t)i);
}

// The transport lookup on given energies and materials: out [n][3] = Sigma_t,
// Sigma_a and nuSigma_f (0 without a nu-fission channel), NaN for an invalid
// material or energy; cum2 [n][stride] receives the running sums.
template <bool NF>
__global__ void k_debug_transport_xs(Tables t, int64_t n, const double* __restrict__ E,
                                     const int32_t* __restrict__ mat, float2* __restrict__ cum2,
                                     int64_t stride, double* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t m = mat[i];
        const double e = E[i];
        double st = __longlong_as_double(0x7ff8000000000000LL), sa = st, nf = st;
        if (m >= 0 && m < t.n_materials && e == e) {
            nf = 0.0;
            macro_transport_pair<NF>(t, m, e, st, sa, cum2 + i * stride, &nf);
        }
        out[3 * i] = st;
        out[3 * i + 1] = sa;
        out[3 * i + 2] = nf;
    }
}

int launch_debug_transport_xs(const Tables& t, int64_t n, const double* E, const int32_t* mat, float2* cum2,
                              int64_t stride, double* out, cudaStream_t st)
{
    const int grid = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    if (t.ch_nu_fission >= 0)
        k_debug_transport_xs<true><<<grid > 0 ? grid : 1, 256, 0, st>>>(t, n, E, mat, cum2, stride, out);
    else
        k_debug_transport_xs<false><<<grid > 0 ? grid : 1, 256, 0, st>>>(t, n, E, mat, cum2, stride, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

__global__ void k_debug_neg_log(const double* __restrict__ x, int64_t n, double* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        out[2 * i] = neg_log_uniform(x[i]);
        out[2 * i + 1] = -log(x[i]);
    }
}

int launch_debug_neg_log(const double* x, int64_t n, double* out, cudaStream_t st)
{
    k_init_nlog<<<1, 256, 0, st>>>();
    const int grid = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    k_debug_neg_log<<<grid > 0 ? grid : 1, 256, 0, st>>>(x, n, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_debug_uniforms(uint2 key, uint64_t hist, uint32_t first, int64_t n, double* out,
                          cudaStream_t st)
{
    const int grid = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    k_debug_uniforms<<<grid > 0 ? grid : 1, 256, 0, st>>>(key, hist, first, n, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

MCX_BOUNDS_READER(bounds_error_transport)

}  // namespace mcx
