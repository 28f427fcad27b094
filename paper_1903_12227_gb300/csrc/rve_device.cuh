// rve_device.cuh -- device-side building blocks of librve (sm_103a).
//
// * complex helpers on float2 / double2;
// * DotAcc: per-thread dot-product accumulators.  FP64 data accumulate in
//   double.  FP32 data: each thread sums its own <= 32 products in FP32, the
//   block combines the thread sums in double-float and the blocks are
//   combined in FP64 -- no long FP32 sums and no per-element FP64 work;
// * deterministic warp / block reductions (fixed tree order);
// * a register-resident Stockham FFT of length n = 2^p (radix 8, then 4 or
//   2) with one padded shared-memory buffer per sequence, used for the
//   separable transforms of the preconditioner;
// * the Hartley "pair" post-processing: the complex DFT Z of a + i b (a, b
//   real) gives the Hartley transforms of a and b, because
//   H_a(k) = Re A_k - Im A_k with A_k = (Z_k + conj Z_{-k}) / 2, and the
//   same for b with B_k = (Z_k - conj Z_{-k}) / 2i.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rve {

// ---------------------------------------------------------------- types --
template <typename V> struct ScalarOf;
template <> struct ScalarOf<float2> { typedef float T; };
template <> struct ScalarOf<double2> { typedef double T; };

template <typename V> __device__ __forceinline__ V mk(typename ScalarOf<V>::T x,
                                                       typename ScalarOf<V>::T y);
template <> __device__ __forceinline__ float2 mk<float2>(float x, float y) { return make_float2(x, y); }
template <> __device__ __forceinline__ double2 mk<double2>(double x, double y) { return make_double2(x, y); }

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { V r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { V r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    V r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// multiply by -i: (x + iy)(-i) = y - ix
template <typename V> __device__ __forceinline__ V cmul_mi(V a) { V r; r.x = a.y; r.y = -a.x; return r; }

// ------------------------------------------------- asynchronous copies --
// One element global -> shared without passing through registers
// (cp.async; 8-byte elements through L1, 16-byte ones bypassing it), the
// commit of the copies issued so far as one group, and the wait until at
// most N groups of this thread are still in flight.
__device__ __forceinline__ void cp_async_v(float2* dst, const float2* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_v(double2* dst, const double2* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
// Asks for `bytes` at `src` to be brought into L2 (no registers, no
// completion to wait for).  src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void prefetch_l2(const void* src, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(src), "r"(bytes) : "memory");
}

// ------------------------------------------------------- dot accumulator --
template <typename T> struct DotAcc;

template <> struct DotAcc<double> {
    double s;
    __device__ __forceinline__ DotAcc() : s(0.0) {}
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};

// FP32 data: a thread sums only its own few (<= 32) products, with fused
// multiply-adds in FP32; the block then combines the per-thread sums in
// double-float (TwoSum, see block_sum2) and the blocks are combined in FP64,
// so no sum longer than 32 terms is formed in FP32.  (hi, lo) is the
// double-float pair of the block tree; lo stays 0 within a thread.
template <> struct DotAcc<float> {
    float hi, lo;
    __device__ __forceinline__ DotAcc() : hi(0.f), lo(0.f) {}
    __device__ __forceinline__ void add(float a, float b) { hi = fmaf(a, b, hi); }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// --------------------------------------------------- deterministic reduce --
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of `v` over the block in a fixed order; result valid in thread 0.
// `scratch` holds at least blockDim.x/32 doubles.  Ends with a barrier so
// that scratch can be reused.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < nw ? scratch[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

// Block sums of two dot-product accumulators; (sx, sy) valid in thread 0.
// FP64 data: double tree.  FP32 data: the whole tree stays in double-float
// (TwoSum on (hi, lo) pairs, fixed xor-butterfly order) and only thread 0
// converts to double, so the block issues a handful of FP64 instructions
// instead of a few per thread (GB300's FP64 pipe is ~1/64 of FP32).
// `scratch` holds 64 floats / 32 doubles.  Contains barriers; ends with one.
__device__ __forceinline__ void df_add(float& hi, float& lo, float oh, float ol) {
    const float t = hi + oh;
    const float bv = t - hi;
    const float e = (hi - (t - bv)) + (oh - bv);
    hi = t;
    lo = lo + ol + e;
}

__device__ __forceinline__ void df_warp(float& hi, float& lo) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
        const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
        df_add(hi, lo, oh, ol);
    }
}

__device__ __forceinline__ void block_sum2(const DotAcc<float>& ax, const DotAcc<float>& ay,
                                           void* scratch, double& sx, double& sy) {
    float* sh = static_cast<float*>(scratch);   // [32][4]
    float xh = ax.hi, xl = ax.lo, yh = ay.hi, yl = ay.lo;
    df_warp(xh, xl);
    df_warp(yh, yl);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    if (lane == 0) {
        sh[4 * wid + 0] = xh; sh[4 * wid + 1] = xl;
        sh[4 * wid + 2] = yh; sh[4 * wid + 3] = yl;
    }
    __syncthreads();
    if (wid == 0) {
        xh = lane < nw ? sh[4 * lane + 0] : 0.f;
        xl = lane < nw ? sh[4 * lane + 1] : 0.f;
        yh = lane < nw ? sh[4 * lane + 2] : 0.f;
        yl = lane < nw ? sh[4 * lane + 3] : 0.f;
        df_warp(xh, xl);
        df_warp(yh, yl);
        if (lane == 0) {
            sx = (double)xh + (double)xl;
            sy = (double)yh + (double)yl;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void block_sum2(const DotAcc<double>& ax, const DotAcc<double>& ay,
                                           void* scratch, double& sx, double& sy) {
    double* sh = static_cast<double*>(scratch);   // [32]
    const double a = block_sum(ax.value(), sh);
    const double b = block_sum(ay.value(), sh);
    if (threadIdx.x == 0) { sx = a; sy = b; }
}

// Fixed-order sum of `count` doubles at src[k*stride] by one warp; every
// lane gets the result.  Plain (coherent) loads: the persistent solver reads
// partial sums written by other blocks earlier in the same launch.
__device__ __forceinline__ double warp_sum_array(const double* src, int count, int stride) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int k = lane; k < count; k += 32) s += src[(int64_t)k * stride];
    return warp_sum(s);
}

// ---------------------------------------------------------- double-word --
// A value carried as the unevaluated sum hi + lo of two floats, for the
// mixed path's true residual, which must be accurate far beyond FP32 but
// must not run on GB300's narrow FP64 pipe.  Built from the error-free
// transformations TwoSum (Knuth), Fast2Sum (Dekker; |a| >= |b| or a = 0) and
// TwoProd with a fused multiply-add, combined as in Dekker (1971) and Joldes,
// Muller & Popescu (ACM TOMS 44, 2017).  The _rn intrinsics keep the compiler
// from contracting or reassociating any step, so every kernel that evaluates
// the same expression gets the same bits.
struct dword { float hi, lo; };

__device__ __forceinline__ dword two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ dword fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// Double-word + double-word ("sloppy" sum): absolute error O(eps^2 (|x|+|y|)),
// which is all a residual needs (its terms cancel; the error budget is set by
// their magnitudes, not by the result's).
__device__ __forceinline__ dword dw_add(dword x, dword y) {
    const dword s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
// Double-word + float.
__device__ __forceinline__ dword dw_add(dword x, float y) {
    const dword s = two_sum(x.hi, y);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}
__device__ __forceinline__ dword dw_neg(dword x) { return {-x.hi, -x.lo}; }
// Exact scaling by a power of two.
__device__ __forceinline__ dword dw_scale2(dword x, float p2) { return {x.hi * p2, x.lo * p2}; }
// Nearest double-word of a double (three FP64 instructions).
__device__ __forceinline__ dword dw_of(double a) {
    const float h = __double2float_rn(a);
    return {h, __double2float_rn(a - (double)h)};
}

// Double word times float: unevaluated (exact high product, error + cross term).
__device__ __forceinline__ dword dw_mulf(dword x, float f) {
    const float p = __fmul_rn(x.hi, f);
    return {p, __fmaf_rn(x.lo, f, __fmaf_rn(x.hi, f, -p))};
}

// Double word of a double from its IEEE-754 fields, with integer
// instructions only: hi = x truncated to float's 24 significant bits
// (exact), lo = the remaining 29 bits rounded to float, so hi + lo carries
// 48+ bits and |lo| < ulp(hi).  |x| below 2^-126 gives (0, 0); the low part
// of |x| below 2^-74 is dropped; |x| beyond float's range gives +-inf.
__device__ __forceinline__ dword dw_split(double x) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(bits >> 63) << 31;
    const int e = (int)((bits >> 52) & 0x7FF);
    const unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
    if (e < 897) return {__int_as_float((int)sign), 0.f};              // zero, tiny
    if (e > 1150) return {__int_as_float((int)(sign | 0x7F800000u | (e == 0x7FF && m ? 0x400000u : 0u))), 0.f};
    const float hi = __int_as_float((int)(sign | ((unsigned)(e - 896) << 23) | (unsigned)(m >> 29)));
    const int pe = e - 948;                    // biased exponent of 2^(e - 1075)
    float lo = 0.f;
    if (pe >= 1) lo = __uint2float_rn((unsigned)(m & 0x1FFFFFFFull)) * __int_as_float(pe << 23);
    return {hi, sign ? -lo : lo};
}

// Double word times double word, unevaluated: exact product of the high
// parts plus its error and the cross terms (the lo*lo term is below eps^2).
__device__ __forceinline__ dword dw_mul(dword x, dword y) {
    const float p = __fmul_rn(x.hi, y.hi);
    return {p, __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, __fmaf_rn(x.hi, y.hi, -p)))};
}

// Per-thread running double-word sum of unevaluated terms (hi, lo).
__device__ __forceinline__ void dw_acc(dword& s, dword t) {
    const dword u = two_sum(s.hi, t.hi);
    s.hi = u.hi;
    s.lo = __fadd_rn(s.lo, __fadd_rn(u.lo, t.lo));
}

// Running sum  s0 + sum_k (+-) c_k w_k  of double-word products: the
// product of the high parts is split exactly (TwoProd) and added with TwoSum;
// the rounding errors and the cross terms gather in a float compensation
// term (the compensated dot product "Dot2" of Ogita, Rump & Oishi, SIAM J.
// Sci. Comput. 26, 2005, with double-word operands).  The error is
// O(eps) |result| + O(eps^2) sum |c_k w_k|.
struct DotDW {
    float s, comp;
    __device__ __forceinline__ explicit DotDW(dword s0) : s(s0.hi), comp(s0.lo) {}
    __device__ __forceinline__ void add(dword a, float whi, float wlo) {
        const float p = __fmul_rn(a.hi, whi);
        const float e = __fmaf_rn(a.hi, whi, -p);
        const float x = __fmaf_rn(a.hi, wlo, __fmaf_rn(a.lo, whi, e));
        const dword t = two_sum(s, p);
        s = t.hi;
        comp = __fadd_rn(comp, __fadd_rn(t.lo, x));
    }
    // the same with a weight that is a single float (a double word with a
    // zero low part, without its zero products)
    __device__ __forceinline__ void add(float a, float whi, float wlo) {
        const float p = __fmul_rn(a, whi);
        const float e = __fmaf_rn(a, whi, -p);
        const float x = __fmaf_rn(a, wlo, e);
        const dword t = two_sum(s, p);
        s = t.hi;
        comp = __fadd_rn(comp, __fadd_rn(t.lo, x));
    }
    __device__ __forceinline__ float value() const { return __fadd_rn(s, comp); }
};

// ------------------------------------------------------- double-double --
// The same error-free transformations on FP64 pairs: a value hi + lo with
// |lo| <= ulp(hi)/2 carries ~106 significant bits.  Used where an FP64 result
// must be accurate to the last bit or beyond (the FP64 A_hom reduction,
// whose low part lets a caller difference two nearby values of A_hom).  The
// _rn intrinsics keep every step as written (no contraction).
struct ddouble { double hi, lo; };

__device__ __forceinline__ ddouble dd_two_sum(double a, double b) {
    const double s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    return {s, __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb))};
}
__device__ __forceinline__ ddouble dd_fast_two_sum(double a, double b) {
    const double s = __dadd_rn(a, b);
    return {s, __dsub_rn(b, __dsub_rn(s, a))};
}
// Accurate sum (Joldes, Muller & Popescu 2017, "AccurateDWPlusDW"): relative
// error O(eps^2) even under cancellation.  Commutative bit for bit, so the
// xor butterflies below leave every lane with the same value.
__device__ __forceinline__ ddouble dd_add(ddouble x, ddouble y) {
    const ddouble s = dd_two_sum(x.hi, y.hi);
    const ddouble t = dd_two_sum(x.lo, y.lo);
    const ddouble v = dd_fast_two_sum(s.hi, __dadd_rn(s.lo, t.hi));
    return dd_fast_two_sum(v.hi, __dadd_rn(t.lo, v.lo));
}
__device__ __forceinline__ ddouble dd_add(ddouble x, double y) {
    const ddouble s = dd_two_sum(x.hi, y);
    return dd_fast_two_sum(s.hi, __dadd_rn(x.lo, s.lo));
}
// Exact difference of two doubles.
__device__ __forceinline__ ddouble dd_sub(double a, double b) { return dd_two_sum(a, -b); }
__device__ __forceinline__ ddouble dd_neg(ddouble x) { return {-x.hi, -x.lo}; }
// Exact scaling by a power of two.
__device__ __forceinline__ ddouble dd_scale2(ddouble x, double p2) {
    return {__dmul_rn(x.hi, p2), __dmul_rn(x.lo, p2)};
}
// Product (TwoProd of the high parts by a fused multiply-add, cross terms
// added; relative error O(eps^2)).
__device__ __forceinline__ ddouble dd_mul(ddouble x, ddouble y) {
    const double p = __dmul_rn(x.hi, y.hi);
    const double e = __fma_rn(x.hi, y.hi, -p);
    const double c = __fma_rn(x.hi, y.lo, __fma_rn(x.lo, y.hi, e));
    return dd_fast_two_sum(p, c);
}
__device__ __forceinline__ ddouble dd_mul(ddouble x, double y) {
    const double p = __dmul_rn(x.hi, y);
    const double e = __fma_rn(x.hi, y, -p);
    return dd_fast_two_sum(p, __fma_rn(x.lo, y, e));
}
// Quotient by a double (one long division step plus a correction).
__device__ __forceinline__ ddouble dd_div(ddouble x, double b) {
    const double q1 = __ddiv_rn(x.hi, b);
    const double p = __dmul_rn(q1, b);
    const double e = __fma_rn(q1, b, -p);
    const double r = __dadd_rn(__dsub_rn(__dsub_rn(x.hi, p), e), x.lo);
    return dd_fast_two_sum(q1, __ddiv_rn(r, b));
}
// Fixed-order butterfly sum over a warp (every lane gets the same value).
__device__ __forceinline__ ddouble dd_warp_sum(ddouble v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const ddouble w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = dd_add(v, w);
    }
    return v;
}

// ------------------------------------------------------------ radix DFTs --
// Forward (exp(-2 pi i rs/R)) in-register DFTs.
template <typename V> __device__ __forceinline__ void dft2(V& a, V& b) {
    V t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <typename V> __device__ __forceinline__ void dft4(V& u0, V& u1, V& u2, V& u3) {
    V s02 = cadd(u0, u2), d02 = csub(u0, u2);
    V s13 = cadd(u1, u3), d13 = cmul_mi(csub(u1, u3));
    u0 = cadd(s02, s13);
    u2 = csub(s02, s13);
    u1 = cadd(d02, d13);
    u3 = csub(d02, d13);
}

template <typename V> __device__ __forceinline__ void dft8(V* u) {
    typedef typename ScalarOf<V>::T T;
    const T c = (T)0.70710678118654752440084436210484903928;
    V e0 = u[0], e1 = u[2], e2 = u[4], e3 = u[6];
    V o0 = u[1], o1 = u[3], o2 = u[5], o3 = u[7];
    dft4(e0, e1, e2, e3);
    dft4(o0, o1, o2, o3);
    // twiddles W8^s = exp(-i pi s/4): 1, c(1-i), -i, -c(1+i)
    V t1 = mk<V>(c * (o1.x + o1.y), c * (o1.y - o1.x));
    V t2 = cmul_mi(o2);
    V t3 = mk<V>(c * (o3.y - o3.x), -c * (o3.x + o3.y));
    u[0] = cadd(e0, o0); u[4] = csub(e0, o0);
    u[1] = cadd(e1, t1); u[5] = csub(e1, t1);
    u[2] = cadd(e2, t2); u[6] = csub(e2, t2);
    u[3] = cadd(e3, t3); u[7] = csub(e3, t3);
}

// ------------------------------------------------ register Stockham FFT --
// Shared-memory index with one spare slot every 16 elements, so that the
// stride-8 output pattern of a radix-8 stage spreads over the banks.
__host__ __device__ __forceinline__ int pidx(int x) { return x + (x >> 4); }

// Distance between consecutive sequences in shared memory: the padded length
// rounded up to 4 (mod 16) elements, so that sequences side by side (columns,
// or the short rows of small grids) start on different banks.
__host__ __device__ __forceinline__ int seq_stride(int n) {
    const int p = n + (n >> 4);
    return p + ((4 - (p & 15)) & 15);
}

// Where the last Stockham stage leaves the transform.
enum { FFT_TO_SMEM = 0, FFT_TO_REGS = 1, FFT_TO_BOTH = 2 };

// Forward DFT (unnormalised) of one sequence of length n = 2^log2n >= 32,
// cooperatively by T = n/8 threads (t in [0, T)).  On entry thread t holds
// v[m] = x[t + m T], m = 0..7 -- exactly the inputs of its butterflies in
// every Stockham stage (one radix-8 butterfly, or two radix-4, or four
// radix-2), so each stage reads its inputs from registers or from `buf`,
// writes its outputs to `buf` (one padded buffer of n elements, see pidx)
// and a barrier separates stages.  The outputs of the last stage fall on the
// same positions t + m T, so they can stay in registers:
//   FFT_TO_SMEM: buf holds X in natural order, then a barrier;
//   FFT_TO_REGS: v[m] = X[t + m T], buf untouched by the last stage, no
//                trailing barrier;
//   FFT_TO_BOTH: both, then a barrier.
// Threads with active == false only take part in the barriers.
// tw[m] = exp(-2 pi i m/n).
// LOG2N > 0 makes the size a compile-time constant: the stages unroll and
// every index folds to an immediate; LOG2N == 0 takes log2n at run time.
// BS: element x of the sequence sits at buf[pidx(x) * BS], so that BS
// sequences can be interleaved element by element (BS consecutive lanes
// working on BS sequences then touch consecutive words).
// The barriers between stages come from `bar` (default: the whole block;
// a row team's own barrier when every row is transformed by its own threads,
// see TeamBar).
struct BlockBar {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
template <int FINAL, int LOG2N = 0, int BS = 1, typename V, typename Bar = BlockBar>
__device__ __forceinline__ void fft_reg(V (&v)[8], V* buf, int log2n_rt, int t,
                                        const V* __restrict__ tw, bool active, Bar bar = Bar()) {
    const int log2n = LOG2N ? LOG2N : log2n_rt;
    const int T = 1 << (log2n - 3);
    const int nstages = (log2n + 2) / 3;   // radix 8, then one radix-4 or -2 tail
#pragma unroll
    for (int stage = 0; stage < (LOG2N ? (LOG2N + 2) / 3 : 4); ++stage) {
        if (!LOG2N && stage >= nstages) break;
        const int log2Ns = 3 * stage;        // every earlier stage was radix 8
        const int rem = log2n - log2Ns;
        const int lr = rem >= 3 ? 3 : rem;
        const int Ns = 1 << log2Ns;
        const int twshift = log2n - log2Ns - lr;
        const bool last = (rem == lr);
        const bool to_smem = !last || FINAL != FFT_TO_REGS;
        const bool to_regs = last && FINAL != FFT_TO_SMEM;
        bar();   // earlier readers of buf are done
        if (active) {
            if (lr == 3) {
                const int k = t & (Ns - 1);
                if (Ns > 1) {
#pragma unroll
                    for (int r = 1; r < 8; ++r) v[r] = cmul(v[r], tw[(r * k) << twshift]);
                }
                dft8(v);   // outputs stay in v[r]: the last stage's slots
                if (to_smem) {
                    const int base = ((t - k) << 3) + k;
#pragma unroll
                    for (int r = 0; r < 8; ++r) buf[pidx(base + r * Ns) * BS] = v[r];
                }
            } else if (lr == 2) {
                V o[8];
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const int j = t + b * T, k = j & (Ns - 1);
                    V a0 = v[b], a1 = v[b + 2], a2 = v[b + 4], a3 = v[b + 6];
                    if (Ns > 1) {
                        a1 = cmul(a1, tw[k << twshift]);
                        a2 = cmul(a2, tw[(2 * k) << twshift]);
                        a3 = cmul(a3, tw[(3 * k) << twshift]);
                    }
                    dft4(a0, a1, a2, a3);
                    o[b] = a0; o[b + 2] = a1; o[b + 4] = a2; o[b + 6] = a3;
                    if (to_smem) {
                        const int base = ((j - k) << 2) + k;
                        buf[pidx(base) * BS] = a0;
                        buf[pidx(base + Ns) * BS] = a1;
                        buf[pidx(base + 2 * Ns) * BS] = a2;
                        buf[pidx(base + 3 * Ns) * BS] = a3;
                    }
                }
                if (to_regs) {
#pragma unroll
                    for (int m = 0; m < 8; ++m) v[m] = o[m];
                }
            } else {
                V o[8];
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int j = t + b * T, k = j & (Ns - 1);
                    V a0 = v[b], a1 = v[b + 4];
                    if (Ns > 1) a1 = cmul(a1, tw[k << twshift]);
                    dft2(a0, a1);
                    o[b] = a0; o[b + 4] = a1;
                    if (to_smem) {
                        const int base = ((j - k) << 1) + k;
                        buf[pidx(base) * BS] = a0;
                        buf[pidx(base + Ns) * BS] = a1;
                    }
                }
                if (to_regs) {
#pragma unroll
                    for (int m = 0; m < 8; ++m) v[m] = o[m];
                }
            }
        }
        if (last) {
            if (FINAL != FFT_TO_REGS) bar();
            break;
        }
        bar();
        if (active) {
#pragma unroll
            for (int m = 0; m < 8; ++m) v[m] = buf[pidx(t + m * T) * BS];
        }
    }
}

// Barrier of the T = n/8 threads that transform one row (a "row team"):
// named barrier 1 + team (T >= 64, a multiple of the warp size; at most four
// teams in a 256-thread block), the warp's own barrier when a team fits in a
// warp (T <= 32: the warp's teams sync together, which is all they need).
struct TeamBar {
    int id, count;
    __device__ __forceinline__ TeamBar(int team, int T) : id(1 + team), count(T) {}
    __device__ __forceinline__ void operator()() const {
        if (count >= 64) asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
        else __syncwarp();
    }
};

// Grid size as compile-time constants (LOG2N > 0) or run-time values (0).
template <int LOG2N> struct Sz {
    static constexpr int log2n = LOG2N, n = 1 << LOG2N, T = (1 << LOG2N) >> 3;
    __device__ __forceinline__ explicit Sz(int) {}
};
template <> struct Sz<0> {
    int log2n, n, T;
    __device__ __forceinline__ explicit Sz(int l) : log2n(l), n(1 << l), T((1 << l) >> 3) {}
};

// Hartley pair from the DFT Z of (a + i b): returns (H_a(k), H_b(k)).
template <typename V> __device__ __forceinline__ V hartley_pair(V zk, V zm) {
    typedef typename ScalarOf<V>::T T;
    const T hf = (T)0.5;
    return mk<V>(hf * ((zk.x + zm.x) - (zk.y - zm.y)), hf * ((zk.y + zm.y) + (zk.x - zm.x)));
}

}  // namespace rve
