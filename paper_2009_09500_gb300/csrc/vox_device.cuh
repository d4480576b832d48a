// vox_device.cuh -- device-side building blocks of libvox (sm_103a).
//
// Small inline-PTX wrappers (global timer, relaxed 64-bit accesses, mbarrier,
// 1-D TMA bulk copy global -> shared) and the per-segment stepping state used by
// the generation kernels.
//
// The stepping state implements Eq. (3) of the paper (G_k = S + W k, W = (E - S)/N)
// with the nearest-lattice rounding done exactly in integers. Per axis a with
// A = |d_a| the voxel offset from S is q(k) = floor((2 k A + N) / (2 N)); the
// remainder r(k) = (2 k A + N) mod 2N then advances by 2A per step and gives back
// 2N, moving the voxel one step along sign(d_a), each time it reaches 2N (A <= N,
// so at most once per step). One division per axis enters a segment mid-way
// (Section 3: voxel k does not depend on voxel k - 1); every further voxel costs
// an add and a compare per minor axis.
#pragma once

#include <cstdint>

namespace vox {

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int32_t ld_volatile_i32(const int32_t *p)
{
    return *reinterpret_cast<const volatile int32_t *>(p);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of an mbarrier, giving up after limit_ns nanoseconds.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
    return true;
}

// 1-D TMA bulk copy global -> this CTA's shared memory; completion is counted in
// bytes on `bar`. dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void set_status(int32_t *status, int32_t code)
{
    atomicCAS(status, 0, code);
}

// ------------------------------------------------------- per-segment stepping
// q = floor(num / den) and r = num - q den for 1 <= den < 2^23 and num / den < 2^22,
// given rcp = 1 / den rounded to nearest in single precision. The quotient is
// estimated as num * rcp in single precision: three roundings (num, the
// reciprocal, the product), each of relative size at most 2^-24, keep the
// estimate within 3 * 2^-24 * 2^22 = 0.75 of num / den, so its integer part is
// q - 1, q or q + 1, and the remainder of that guess (in (-2 den, 2 den), hence
// exact modulo 2^32) settles which: the estimate-and-correct step of long
// division (Knuth, TAOCP vol. 2, 4.3.1), with one correction.
__device__ __forceinline__ void divmod_est(uint64_t num, int32_t den, float rcp, int32_t &q, int32_t &r)
{
    int32_t qq = __float2int_rz(__fmul_rn(__ull2float_rn(num), rcp));
    int32_t rr = static_cast<int32_t>(static_cast<uint32_t>(num) - static_cast<uint32_t>(qq) * static_cast<uint32_t>(den));
    if (rr < 0) {
        --qq;
        rr += den;
    } else if (rr >= den) {
        ++qq;
        rr -= den;
    }
    q = qq;
    r = rr;
}

// Voxel offset q and remainder r of one axis at step k (0 < k <= N < 2^22,
// A <= N, A < 2^21): q = floor((2 k A + N) / (2 N)) <= A, r = (2 k A + N) - 2 N q.
// rcp2N = 1 / (2N) rounded to nearest in single precision.
__device__ __forceinline__ void axis_entry(int32_t A, int32_t N, int32_t k, float rcp2N, int32_t &q, int32_t &r)
{
    if (A == N) {  // the numerator is N (mod 2N) for every k
        q = k;
        r = N;
    } else if (A == 0) {
        q = 0;
        r = N;
    } else {
        divmod_est(2ull * static_cast<uint64_t>(k) * static_cast<uint64_t>(A) + static_cast<uint64_t>(N), 2 * N,
                   rcp2N, q, r);
    }
}

// Output encodings of a voxel (x, y, z).
template <typename PackT>
__device__ __forceinline__ PackT pack_unit(int axis);

template <>
__device__ __forceinline__ uint32_t pack_unit<uint32_t>(int axis)
{
    return 1u << (10 * axis);
}

template <>
__device__ __forceinline__ uint64_t pack_unit<uint64_t>(int axis)
{
    return 1ull << (21 * axis);
}

// Signed step of `unit` along an axis whose delta is d (+unit, -unit or 0),
// in two's complement so that adding it to a packed word moves one field.
template <typename T>
__device__ __forceinline__ T signed_step(int32_t d, T unit)
{
    return d > 0 ? unit : (d < 0 ? static_cast<T>(T(0) - unit) : T(0));
}

// x += y (mod 2^32); returns the carry out of bit 31 (0 or 1).
__device__ __forceinline__ uint32_t add_carry(uint32_t &x, uint32_t y)
{
    uint32_t c;
    asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, 0, 0;" : "+r"(x), "=r"(c) : "r"(y));
    return c;
}

// P += dm + cb db + cc dc (mod 2^bits) for carries cb, cc in {0, 1}: the packed
// word moves one voxel along the major axis and along each minor axis whose
// carry is set. 32-bit words: three integer adds; 64-bit words: one add and two
// multiply-adds by the carry, each chained through the carry flag from the low
// to the high half.
__device__ __forceinline__ void advance_packed(uint32_t &P, uint32_t dm, uint32_t cb, uint32_t db, uint32_t cc,
                                               uint32_t dc)
{
    P += dm + cb * db + cc * dc;
}

__device__ __forceinline__ void advance_packed(uint64_t &P, uint64_t dm, uint32_t cb, uint64_t db, uint32_t cc,
                                               uint64_t dc)
{
    asm("{\n\t.reg .u32 lo, hi;\n\t"
        "mov.b64 {lo, hi}, %0;\n\t"
        "add.cc.u32 lo, lo, %1;\n\t"
        "addc.u32 hi, hi, %2;\n\t"
        "mad.lo.cc.u32 lo, %3, %4, lo;\n\t"
        "madc.lo.u32 hi, %3, %5, hi;\n\t"
        "mad.lo.cc.u32 lo, %6, %7, lo;\n\t"
        "madc.lo.u32 hi, %6, %8, hi;\n\t"
        "mov.b64 %0, {lo, hi};\n\t}"
        : "+l"(P)
        : "r"(static_cast<uint32_t>(dm)), "r"(static_cast<uint32_t>(dm >> 32)), "r"(cb),
          "r"(static_cast<uint32_t>(db)), "r"(static_cast<uint32_t>(db >> 32)), "r"(cc),
          "r"(static_cast<uint32_t>(dc)), "r"(static_cast<uint32_t>(dc >> 32)));
}

// Stepping state of one segment. PackT: uint32_t (LIST32) or uint64_t (LIST64);
// LinT: uint32_t or uint64_t volume bit index (volumes up to or beyond 2^32 bits).
// The three minor/major roles are fixed at entry: the major axis (|d| = N) moves
// every step, the two minor axes move when their remainder r (0 <= r < 2N) plus
// 2|d| reaches 2N. Each r is held biased, as r + 2^32 - 2N (mod 2^32, no wrap for
// r < 2N), so that adding 2|d| carries out of 32 bits exactly when the axis moves.
template <typename PackT, typename LinT>
struct Stepper {
    int32_t left;        // steps still to take inside this segment after entry (N - k)
    uint32_t Ab2, Ac2;   // 2|d| of the two minor axes
    uint32_t eb, ec;     // their biased remainders
    uint32_t bias;       // 2^32 - 2N (mod 2^32)
    PackT P, dPm, dPb, dPc;
    LinT L, dLm, dLb, dLc;

    // Enter segment (x0, y0, z0) -> (x1, y1, z1) at step k (0 <= k <= N).
    __device__ __forceinline__ void enter(const int32_t *rec, int32_t k, LinT w, LinT wh)
    {
        const int32_t x0 = rec[0], y0 = rec[1], z0 = rec[2];
        const int32_t dx = rec[3] - x0, dy = rec[4] - y0, dz = rec[5] - z0;
        const int32_t ax = abs(dx), ay = abs(dy), az = abs(dz);
        const int32_t N = max(ax, max(ay, az));
        left = N - k;
        // major axis: the first with |d| = N; minors b, c are the other two in order
        const bool mx = (ax == N);
        const bool my = !mx && (ay == N);
        const int32_t dm = mx ? dx : (my ? dy : dz);
        const int32_t db = mx ? dy : dx;
        const int32_t dc = (mx || my) ? dz : dy;
        const int axis_m = mx ? 0 : (my ? 1 : 2);
        const int axis_b = mx ? 1 : 0;
        const int axis_c = (mx || my) ? 2 : 1;
        // the major axis is at offset k (remainder N); one division per minor axis
        int32_t qb = 0, qc = 0, rb = N, rc = N;
        if (k > 0) {  // k = 0: every offset is 0 and every remainder N
            const float rcp2N = __frcp_rn(static_cast<float>(2 * N));
            axis_entry(abs(db), N, k, rcp2N, qb, rb);
            axis_entry(abs(dc), N, k, rcp2N, qc, rc);
        }
        const int32_t qx = mx ? k : qb;
        const int32_t qy = my ? k : (mx ? qb : qc);
        const int32_t qz = (mx || my) ? qc : k;
        const int32_t vx = x0 + (dx >= 0 ? qx : -qx);
        const int32_t vy = y0 + (dy >= 0 ? qy : -qy);
        const int32_t vz = z0 + (dz >= 0 ? qz : -qz);
        P = static_cast<PackT>(vx) | (static_cast<PackT>(vy) * pack_unit<PackT>(1)) |
            (static_cast<PackT>(vz) * pack_unit<PackT>(2));
        L = static_cast<LinT>(vx) + static_cast<LinT>(vy) * w + static_cast<LinT>(vz) * wh;
        Ab2 = 2u * static_cast<uint32_t>(abs(db));
        Ac2 = 2u * static_cast<uint32_t>(abs(dc));
        bias = 0u - 2u * static_cast<uint32_t>(N);
        eb = static_cast<uint32_t>(rb) + bias;
        ec = static_cast<uint32_t>(rc) + bias;
        dPm = signed_step<PackT>(dm, pack_unit<PackT>(axis_m));
        dPb = signed_step<PackT>(db, pack_unit<PackT>(axis_b));
        dPc = signed_step<PackT>(dc, pack_unit<PackT>(axis_c));
        const LinT um = axis_m == 0 ? LinT(1) : (axis_m == 1 ? w : wh);
        const LinT ub = axis_b == 0 ? LinT(1) : w;
        const LinT uc = axis_c == 2 ? wh : w;
        dLm = signed_step<LinT>(dm, um);
        dLb = signed_step<LinT>(db, ub);
        dLc = signed_step<LinT>(dc, uc);
    }

    // One step along the segment: the carries say which minor axes move, and a
    // moved axis's remainder is re-biased (r + 2|d| - 2N). Stepping past the last
    // voxel is harmless (the state is simply not used again), so callers may step
    // once too often.
    template <bool kP, bool kL>
    __device__ __forceinline__ void step()
    {
        if (kL) L += dLm;
        const uint32_t cb = add_carry(eb, Ab2);
        const uint32_t cc = add_carry(ec, Ac2);
        eb += cb * bias;
        ec += cc * bias;
        if (kP) advance_packed(P, dPm, cb, dPb, cc, dPc);
        if (kL) L += static_cast<LinT>(cb) * dLb + static_cast<LinT>(cc) * dLc;
    }
};

// int(|d|) for |d|^2 = x < 2^45: a single-precision square root (within a few
// units of the answer for r < 2^22; double precision is a slow pipe on this
// GPU), then corrected with integer comparisons so that r * r <= x < (r + 1)^2
// exactly (the N of Eq. (1)).
__device__ __forceinline__ int32_t isqrt_i64(int64_t x)
{
    int64_t r = static_cast<int64_t>(sqrtf(static_cast<float>(x)));
    while (r > 0 && r * r > x) --r;
    while ((r + 1) * (r + 1) <= x) ++r;
    return static_cast<int32_t>(r);
}

__device__ __forceinline__ int32_t euclid_steps(const int32_t *rec)
{
    int64_t s = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int64_t d = static_cast<int64_t>(rec[3 + a]) - rec[a];
        s += d * d;
    }
    return isqrt_i64(s);
}

// Stepping state with the Euclidean N: no axis moves every step, so all three
// carry (remainder r_a = (2 k A_a + N) mod 2N, the offset growing when it wraps;
// A_a <= N since N = int(|d|) >= max |d_a|). As in Stepper, each r_a is held
// biased by 2^32 - 2N, so that the carry of one add says whether the axis moves.
template <typename PackT, typename LinT>
struct EuclidStepper {
    uint32_t bias;         // 2^32 - 2N (mod 2^32)
    uint32_t A2[3], e[3];  // 2 A_a and the biased remainders
    PackT P, dP[3];
    LinT L, dL[3];

    __device__ __forceinline__ void enter(const int32_t *rec, int32_t k, LinT w, LinT wh)
    {
        enter_n(rec, euclid_steps(rec), k, w, wh);
    }

    // As enter, with N = int(|E - S|) known (a segment's sample count minus one).
    __device__ __forceinline__ void enter_n(const int32_t *rec, int32_t N, int32_t k, LinT w, LinT wh)
    {
        bias = 0u - 2u * static_cast<uint32_t>(N);
        int32_t v[3];
        const float rcp2N = k > 0 ? __frcp_rn(static_cast<float>(2 * N)) : 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int32_t d = rec[3 + a] - rec[a];
            const int32_t A = abs(d);
            int32_t q = 0, rr = N;
            if (k > 0) axis_entry(A, N, k, rcp2N, q, rr);
            e[a] = static_cast<uint32_t>(rr) + bias;
            A2[a] = 2u * static_cast<uint32_t>(A);
            v[a] = rec[a] + (d >= 0 ? q : -q);
            dP[a] = signed_step<PackT>(d, pack_unit<PackT>(a));
            dL[a] = signed_step<LinT>(d, a == 0 ? LinT(1) : (a == 1 ? w : wh));
        }
        P = static_cast<PackT>(v[0]) | (static_cast<PackT>(v[1]) * pack_unit<PackT>(1)) |
            (static_cast<PackT>(v[2]) * pack_unit<PackT>(2));
        L = static_cast<LinT>(v[0]) + static_cast<LinT>(v[1]) * w + static_cast<LinT>(v[2]) * wh;
    }

    // Advance one sample; true when the voxel changed (some axis moved).
    template <bool kP, bool kL>
    __device__ __forceinline__ bool step()
    {
        uint32_t c[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            c[a] = add_carry(e[a], A2[a]);
            e[a] += c[a] * bias;
        }
        if (kP) P += static_cast<PackT>(c[0]) * dP[0] + static_cast<PackT>(c[1]) * dP[1] + static_cast<PackT>(c[2]) * dP[2];
        if (kL) L += static_cast<LinT>(c[0]) * dL[0] + static_cast<LinT>(c[1]) * dL[1] + static_cast<LinT>(c[2]) * dL[2];
        return (c[0] | c[1] | c[2]) != 0u;
    }
};

}  // namespace vox
