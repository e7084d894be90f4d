// kernels.cu -- the multi-cell BDF / modified-Newton solve on sm_103a.
//
// One warp integrates one cell (Implementations section of the paper:
// all cells' data in one structure, the cell loop inside the solver; its
// Conclusions: the whole solver on the GPU).  Per cell:
//   a1  rate constants k~_j(T, P[, J_cell][, theta])         lanes over reactions
//   a2  f(y): rates r_j, then the species-major gather       f program
//   a3/a4  M = I - c J(y_pred) straight into the LU slots    partials + M program
//   a5  static-order sparse LU, forward/back substitution    LU / fwd / bwd programs
//   a6  modified Newton, a7 error test and step/order control, history update
// The cell's sparse working set (LU values, f/J scratch) lives in shared
// memory; per-species vectors and the BDF history live in registers, species
// s = lane + 32 k.  All control decisions are warp-uniform: every lane
// computes the same reductions (butterfly sums are order-symmetric).
//
// FP64 on GB300 issues one warp instruction per 16 SM cycles whether 1 or 32
// lanes are active, so the sparse work is packed into 32-wide passes by the
// host scheduler.  The persistent driver stages the tables every warp reads
// all the time (f and triangular-solve programs, reaction slot tables,
// constants, step-factor grid) into shared memory once per block with a TMA
// bulk copy; the large M and LU programs stream from L2 with a deep prefetch.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "internal.h"
#include "device_common.cuh"

namespace chemgpu {

__constant__ double c_gam[QMAX + 2];
__constant__ double c_igam[QMAX + 2];

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int NEWTON_MAXITER = 3;
constexpr double CRDOWN = 0.3, RDIV = 2.0, DGMAX = 0.3, THRESH = 1.5;   // corrector bound 0.1 (q+1): host table
constexpr int MSBP = 20, MXNEF = 7, MXNCF = 10;
constexpr double ETA_CF = 0.25, ETA_MXF = 0.2, ETA_CST_SAFETY = 0.9, ETA_CST_MIN = 0.1, STRETCH = 1e-3;
constexpr int ORDER_WARPS = 8;          // cells per block of the queue-order kernel

struct SolveParams {
  double rtol, atol, dt;
  int max_order, max_steps;
  int cell_bytes;      // shared memory per warp
  int wd_pad;          // Wd length rounded so WL starts 16-byte aligned
  int warps_per_block;
  int prec;            // 0: FP64 LU, 1: FP32 LU
  int tab_bytes;       // staged table bytes at the start of shared memory (0 if not staged)
  int couple;          // coupled group size (warps_per_block is a multiple of it); 1: independent cells
  long long stage_wait;   // iterations of the first bounded wait for the staged tables
  long long smem_bytes;   // host side: the launch's dynamic shared memory (0: tables + cells)
};

// Reciprocal from the hardware estimate r (relative error e = 1 - x r of
// about 2^-23) refined by one cubically convergent Newton-Raphson step
// (Householder's order-3 iteration for 1/x): r <- r (1 + e + e^2), computed as
// r + r (e + e e) with three FMAs; the step leaves an error of order e^3
// (2^-69), below the final rounding, so the result is within 1 ulp of 1/x
// (and almost always correctly rounded) for normal x with normal 1/x.  Two
// quadratic steps r <- r (2 - x r) would take four FMAs.
__device__ __forceinline__ double recip_nr(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}
__device__ __forceinline__ double lu_recip(double x) { return recip_nr(x); }
__device__ __forceinline__ float lu_recip(float x) { return __frcp_rn(x); }

template <bool SMEM>
__device__ __forceinline__ uint2 ld_op(const ushort4 *p) {
  if (SMEM) return *reinterpret_cast<const uint2 *>(p);
  return __ldg(reinterpret_cast<const uint2 *>(p));
}

template <typename T>
__device__ __forceinline__ T &at(unsigned char *base, unsigned off) {
  return *reinterpret_cast<T *>(base + off);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory accesses by 32-bit shared address (the work arrays always live in shared memory)
__device__ __forceinline__ double lds(double *, uint32_t a) {
  double v;
  asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ float lds(float *, uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void sts(uint32_t a, double v) { asm volatile("st.shared.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory"); }
__device__ __forceinline__ void sts(uint32_t a, float v) { asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory"); }

// Run a warp program (byte-offset ops, see internal.h) over the work array W,
// the next pass's op prefetched.  The loop is deliberately not unrolled and
// prefetches one pass only: the solve kernel is bound by instruction fetch as
// much as by latency, and deeper prefetch (unrolled copies of the pass body at
// every call site) measured 17% slower on the persistent driver and 33% on the
// plain one.  Calls out of line measured slower still (register save/restore).
template <typename T, bool NEG, bool SMEM>
__device__ __forceinline__ void run_ops(const ushort4 *ops, const int np, T *W, const int lane) {
  const uint32_t wb = smem_addr(W);
  T *const tag = nullptr;
  ops += lane;
  uint2 next = np > 0 ? ld_op<SMEM>(ops) : make_uint2(0, 0);   // packed: x = t | a << 16, y = b | c << 16
#pragma unroll 1
  for (int p = 0; p < np; ++p) {
    const uint2 op = next;
    if (p + 1 < np) next = ld_op<SMEM>(ops + (size_t)(p + 1) * WARP);
    const uint32_t ot = op.x & 0xffff, oa = op.x >> 16, ob = op.y & 0xffff, oc = op.y >> 16;
    if (oc == DEV_RECIP) {
      sts(wb + ot, -lu_recip(lds(tag, wb + oa)));
    } else {
      const T a = lds(tag, wb + oa), b = lds(tag, wb + ob), c = lds(tag, wb + oc);
      sts(wb + ot, NEG ? fma(-a, b, c) : fma(a, b, c));
    }
    __syncwarp();
  }
}

// The same interpreter for programs in global memory, with the ops streamed
// RING passes ahead by cp.async into a ring of RING x 256 bytes of shared
// memory (ring: 8-byte aligned shared address).  Each lane copies and reads
// only its own op slots, so cp.async.wait_group alone orders them.
__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// The next pass's op is read from the ring one pass ahead, so that shared-memory
// load overlaps the current pass (the ring slot it reuses held the op read two
// passes earlier).
template <typename T, bool NEG, int RING>
__device__ __forceinline__ void run_ops_ring(const ushort4 *ops, const int np, T *W, const int lane, const uint32_t ring) {
  const uint32_t wb = smem_addr(W);
  T *const tag = nullptr;
  const uint2 *g = reinterpret_cast<const uint2 *>(ops) + lane;
  const uint32_t rb = ring + 8u * lane;
#pragma unroll 1
  for (int i = 0; i < RING - 1; ++i) {
    if (i < np) cp_async8(rb + 256u * i, g + (size_t)i * WARP);
    cp_async_commit();
  }
  cp_async_wait<RING - 2>();            // pass 0's group has landed
  uint32_t nx = 0, ny = 0;
  if (np > 0) asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(nx), "=r"(ny) : "r"(rb) : "memory");
#pragma unroll 1
  for (int p = 0; p < np; ++p) {
    const uint32_t ox = nx, oy = ny;
    const int q = p + RING - 1;
    if (q < np) cp_async8(rb + 256u * (q % RING), g + (size_t)q * WARP);
    cp_async_commit();
    cp_async_wait<RING - 2>();          // pass p+1's group has landed
    if (p + 1 < np)
      asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(nx), "=r"(ny) : "r"(rb + 256u * ((p + 1) % RING)) : "memory");
    const uint32_t ot = ox & 0xffff, oa = ox >> 16, ob = oy & 0xffff, oc = oy >> 16;
    if (oc == DEV_RECIP) {
      sts(wb + ot, -lu_recip(lds(tag, wb + oa)));
    } else {
      const T a = lds(tag, wb + oa), b = lds(tag, wb + ob), c = lds(tag, wb + oc);
      sts(wb + ot, NEG ? fma(-a, b, c) : fma(a, b, c));
    }
    __syncwarp();
  }
  cp_async_wait<0>();                   // nothing in flight once the ring's memory is reused
}

// One FMA op / a pair of independent FMA ops / a reciprocal op of a lane
// (packed ops: x = t | a << 16, y = b | c << 16, byte offsets into W at wb).
template <typename T, bool NEG>
__device__ __forceinline__ void op_fma(uint32_t wb, uint2 o) {
  T *const tag = nullptr;
  const T a = lds(tag, wb + (o.x >> 16)), b = lds(tag, wb + (o.y & 0xffff)), c = lds(tag, wb + (o.y >> 16));
  sts(wb + (o.x & 0xffff), NEG ? fma(-a, b, c) : fma(a, b, c));
}
template <typename T, bool NEG>
__device__ __forceinline__ void op_fma2(uint32_t wb, uint2 o, uint2 u) {
  T *const tag = nullptr;
  const T a = lds(tag, wb + (o.x >> 16)), b = lds(tag, wb + (o.y & 0xffff)), c = lds(tag, wb + (o.y >> 16));
  const T a2 = lds(tag, wb + (u.x >> 16)), b2 = lds(tag, wb + (u.y & 0xffff)), c2 = lds(tag, wb + (u.y >> 16));
  sts(wb + (o.x & 0xffff), NEG ? fma(-a, b, c) : fma(a, b, c));
  sts(wb + (u.x & 0xffff), NEG ? fma(-a2, b2, c2) : fma(a2, b2, c2));
}
// A lane of a pass with reciprocals: W[t] = -1/W[a] (c == DEV_RECIP) or an
// FMA, without a branch.  FP64: every lane forms the estimate r of 1/W[a] and
// the cubic step's e = 1 - x r, e + e^2 (recip_nr), and the final FMA is
// fma(-r, e + e^2, -r) = -recip_nr(x) in a reciprocal lane, the op's own FMA
// in the others (whose r and e are discarded).
template <typename T, bool NEG>
__device__ __forceinline__ void op_mixed(uint32_t wb, uint2 o);
template <>
__device__ __forceinline__ void op_mixed<double, false>(uint32_t wb, uint2 o) {
  double *const tag = nullptr;
  const uint32_t oa = o.x >> 16, oc = o.y >> 16;
  const bool rcp = oc == DEV_RECIP;
  const double x = lds(tag, wb + oa), b = lds(tag, wb + (rcp ? oa : (o.y & 0xffff))), c = lds(tag, wb + (rcp ? oa : oc));
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  const double ee = fma(e, e, e);
  sts(wb + (o.x & 0xffff), rcp ? fma(-r, ee, -r) : fma(x, b, c));
}
template <>
__device__ __forceinline__ void op_mixed<float, false>(uint32_t wb, uint2 o) {
  float *const tag = nullptr;
  const uint32_t oa = o.x >> 16, oc = o.y >> 16;
  const bool rcp = oc == DEV_RECIP;
  const float x = lds(tag, wb + oa), b = lds(tag, wb + (rcp ? oa : (o.y & 0xffff))), c = lds(tag, wb + (rcp ? oa : oc));
  sts(wb + (o.x & 0xffff), rcp ? -__frcp_rn(x) : fmaf(x, b, c));
}

// A program with a run table (RUN_* units, internal.h).  The ops of the next
// two passes are held in registers (n0, n1) and refilled as the units consume
// them, so a unit never waits for its own ops.  Runs are read from shared
// memory (SMEM) or global memory like the ops; WIDE / RECIP: the program has
// pair / reciprocal units (a run table without them compiles to a plain loop).
template <typename T, bool NEG, bool SMEM, bool WIDE, bool RECIP>
__device__ __forceinline__ void run_prog(const ushort4 *ops, const uint32_t *runs, const int nruns, const int np, T *W,
                                         const int lane) {
  const uint32_t wb = smem_addr(W);
  ops += lane;
  uint2 n0 = np > 0 ? ld_op<SMEM>(ops) : make_uint2(0, 0);
  uint2 n1 = np > 1 ? ld_op<SMEM>(ops + WARP) : make_uint2(0, 0);
  int p = 0;
#pragma unroll 1
  for (int r = 0; r < nruns; ++r) {
    const uint32_t rr = SMEM ? runs[r] : __ldg(runs + r);
    const uint32_t kind = rr >> 28;
    int n = (int)(rr & 0x0fffffffu);
    if (WIDE && kind == RUN_FMA2) {
#pragma unroll 1
      for (; n > 0; --n, p += 2) {
        const uint2 o = n0, u = n1;
        if (p + 2 < np) n0 = ld_op<SMEM>(ops + (size_t)(p + 2) * WARP);
        if (p + 3 < np) n1 = ld_op<SMEM>(ops + (size_t)(p + 3) * WARP);
        op_fma2<T, NEG>(wb, o, u);
        __syncwarp();
      }
    } else if (RECIP && kind == RUN_RECIP) {
#pragma unroll 1
      for (; n > 0; --n, ++p) {
        const uint2 o = n0;
        n0 = n1;
        if (p + 2 < np) n1 = ld_op<SMEM>(ops + (size_t)(p + 2) * WARP);
        op_mixed<T, NEG>(wb, o);
        __syncwarp();
      }
    } else {
#pragma unroll 1
      for (; n > 0; --n, ++p) {
        const uint2 o = n0;
        n0 = n1;
        if (p + 2 < np) n1 = ld_op<SMEM>(ops + (size_t)(p + 2) * WARP);
        op_fma<T, NEG>(wb, o);
        __syncwarp();
      }
    }
  }
}

// The same for programs in global memory, the ops streamed through a ring of
// RING x 256 bytes of shared memory (ring: 8-byte aligned shared address) as
// in run_ops_ring.  Invariant at the start of a unit at pass p: passes up to
// p + RING - 3 are issued and the ops of passes p and p + 1 are in n0, n1.  A
// unit issues one pass per pass it consumes, into the slots of passes p - 2
// (and p - 1), whose ops were read into registers and used by earlier units;
// it then waits until pass p + 2 (and p + 3) has landed and refills n0, n1.
template <typename T, bool NEG, int RING, bool WIDE, bool RECIP>
__device__ __forceinline__ void run_prog_ring(const ushort4 *ops, const uint32_t *runs, const int nruns, const int np, T *W,
                                              const int lane, const uint32_t ring) {
  static_assert(RING >= 6, "ring too shallow to run ahead");
  const uint32_t wb = smem_addr(W);
  const uint2 *g = reinterpret_cast<const uint2 *>(ops) + lane;
  const uint32_t rb = ring + 8u * lane;
#pragma unroll 1
  for (int i = 0; i < RING - 2; ++i) {
    if (i < np) cp_async8(rb + 256u * i, g + (size_t)i * WARP);
    cp_async_commit();
  }
  cp_async_wait<RING - 4>();            // passes 0 and 1 have landed
  uint2 n0 = make_uint2(0, 0), n1 = make_uint2(0, 0);
  if (np > 0) asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(n0.x), "=r"(n0.y) : "r"(rb) : "memory");
  if (np > 1) asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(n1.x), "=r"(n1.y) : "r"(rb + 256u) : "memory");
  int p = 0;
#pragma unroll 1
  for (int r = 0; r < nruns; ++r) {
    const uint32_t rr = __ldg(runs + r);
    const uint32_t kind = rr >> 28;
    int n = (int)(rr & 0x0fffffffu);
    if (WIDE && kind == RUN_FMA2) {
#pragma unroll 1
      for (; n > 0; --n, p += 2) {
        const uint2 o = n0, u = n1;
        const int q = p + RING - 2;
        if (q < np) cp_async8(rb + 256u * (q % RING), g + (size_t)q * WARP);
        cp_async_commit();
        if (q + 1 < np) cp_async8(rb + 256u * ((q + 1) % RING), g + (size_t)(q + 1) * WARP);
        cp_async_commit();
        cp_async_wait<RING - 4>();      // passes p + 2 and p + 3 have landed
        if (p + 2 < np)
          asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(n0.x), "=r"(n0.y) : "r"(rb + 256u * ((p + 2) % RING)) : "memory");
        if (p + 3 < np)
          asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(n1.x), "=r"(n1.y) : "r"(rb + 256u * ((p + 3) % RING)) : "memory");
        op_fma2<T, NEG>(wb, o, u);
        __syncwarp();
      }
    } else {
#pragma unroll 1
      for (; n > 0; --n, ++p) {
        const uint2 o = n0;
        n0 = n1;
        const int q = p + RING - 2;
        if (q < np) cp_async8(rb + 256u * (q % RING), g + (size_t)q * WARP);
        cp_async_commit();
        cp_async_wait<RING - 4>();      // pass p + 2 has landed
        if (p + 2 < np)
          asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(n1.x), "=r"(n1.y) : "r"(rb + 256u * ((p + 2) % RING)) : "memory");
        if (RECIP && kind == RUN_RECIP) op_mixed<T, NEG>(wb, o);
        else op_fma<T, NEG>(wb, o);
        __syncwarp();
      }
    }
  }
  cp_async_wait<0>();                   // nothing in flight once the ring's memory is reused
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(FULL, v, o));
  return v;
}

// Comparisons of non-negative doubles on the integer pipe.  FP64 compares,
// min/max and conversions issue on the FP64 pipe at the cost of an FMA or more
// (one warp instruction per 64 cycles of an SM sub-partition); the IEEE bit
// patterns of +0 .. +inf order as the numbers do, and a NaN of either sign
// compares above +inf as an unsigned integer, so these give the FP results
// for operands >= +0 or NaN.
constexpr unsigned long long INF_BITS = 0x7ff0000000000000ull, ABS_MASK = 0x7fffffffffffffffull;
__device__ __forceinline__ unsigned long long ubits(double x) { return (unsigned long long)__double_as_longlong(x); }
// a <= b (false if either is NaN)
__device__ __forceinline__ bool le_nn(double a, double b) {
  const unsigned long long ua = ubits(a), ub = ubits(b);
  return ua <= ub && ub <= INF_BITS;
}
// a > b (false if either is NaN)
__device__ __forceinline__ bool gt_nn(double a, double b) {
  const unsigned long long ua = ubits(a), ub = ubits(b);
  return ua > ub && ua <= INF_BITS;
}
// max(a, b) (a, b >= +0, not NaN)
__device__ __forceinline__ double max_nn(double a, double b) { return ubits(a) >= ubits(b) ? a : b; }
// a == b for any doubles (false if NaN; +0 and -0 are equal)
__device__ __forceinline__ bool eq_fp(double a, double b) {
  const unsigned long long ua = ubits(a), ub = ubits(b);
  return (ua == ub && (ua & ABS_MASK) <= INF_BITS) || ((ua | ub) & ABS_MASK) == 0;
}
// x < 0 (false for -0 and NaN; true for -inf)
__device__ __forceinline__ bool lt0(double x) {
  const unsigned long long u = ubits(x), a = u & ABS_MASK;
  return u != a && a != 0 && a <= INF_BITS;
}

// Warp sum of non-negative doubles on the integer pipe (the five FP64 adds of
// the butterfly cost 64 cycles of an SM sub-partition each): every lane's term
// s = m 2^(e - 1075) (m the 53-bit significand, e the biased exponent) becomes
// the integer F = m 2^(5 + e - emax), emax the largest exponent in the warp,
// truncated (F < 2^58); the 32 F are summed exactly as three 27-bit limbs
// (redux.sync.add: 32 terms below 2^27 fit 32 bits) and the total rounded once
// to nearest even.  A truncated term loses less than 1/32 of an ulp of the
// largest term, so the result is within 1.5 ulp of the exact sum (the
// butterfly's five roundings, 2.5).  Terms below 2^-1022 (subnormal) are
// dropped: with emax >= 64 they are below 2^-63 of the largest.  A warp with an
// infinite, NaN or negative term, or with every term below 2^-959, takes the
// FP64 butterfly.
__device__ __forceinline__ double warp_sum_nn(double s) {
  constexpr unsigned long long FRAC = 0x000fffffffffffffull, ONE53 = 1ull << 52;
  const unsigned long long u = ubits(s);
  const unsigned e = (unsigned)(u >> 52);
  const unsigned emax = __reduce_max_sync(FULL, e);
  if (emax >= 0x7ffu || emax < 64u) return warp_sum(s);
  const unsigned sh = emax - e;
  unsigned long long F = 0;
  if (e != 0 && sh < 64u) F = (((u & FRAC) | ONE53) << 5) >> sh;
  const unsigned s0 = __reduce_add_sync(FULL, (unsigned)F & 0x7ffffffu);
  const unsigned s1 = __reduce_add_sync(FULL, (unsigned)(F >> 27) & 0x7ffffffu);
  const unsigned s2 = __reduce_add_sync(FULL, (unsigned)(F >> 54));
  const unsigned long long tot =
      (unsigned long long)s0 + ((unsigned long long)s1 << 27) + ((unsigned long long)s2 << 54);
  // tot >= 2^57 (a lane with e == emax holds m 2^5), tot < 2^63
  const int b = 63 - __clzll((long long)tot);
  const int r = b - 52;
  unsigned long long mant = tot >> r;
  const unsigned long long rem = tot & ((1ull << r) - 1ull), half = 1ull << (r - 1);
  if (rem > half || (rem == half && (mant & 1ull))) ++mant;
  int E = (int)emax + b - 57;          // the sum is tot 2^(emax - 1080)
  if (mant >> 53) {
    mant >>= 1;
    ++E;
  }
  if (E >= 0x7ff) return __longlong_as_double((long long)INF_BITS);
  return __longlong_as_double((long long)(((unsigned long long)E << 52) | (mant & FRAC)));
}

// Index i of the largest step factor g_i of the grid 2^(i/8) (shifted so the
// smallest is index 0) whose threshold (host table row p, decreasing in i)
// the squared-norm sum e meets; 0 if none.  The thresholds are scaled on the
// host so that the raw warp sum is compared (e >= +0 or NaN; NaN meets none).
__device__ __forceinline__ int grid_idx(const double *thr, double e, int p, int lane) {
  const double *tp = thr + p * GRID_N;
  const bool ok0 = le_nn(e, tp[lane]);
  const bool ok1 = (lane + WARP < GRID_N) && le_nn(e, tp[lane + WARP]);
  const int cnt = __popc(__ballot_sync(FULL, ok0)) + __popc(__ballot_sync(FULL, ok1));
  return cnt > 0 ? cnt - 1 : 0;
}

// ------------------------------------------------------------- TMA staging

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// bounded wait for phase `parity` of the barrier; false if the limit ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit) {
  for (long long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Table bases of one block: base holds the hot prefix (programs and slots used
// every Newton iteration), staged in shared memory or the blob in global
// memory; gbase is always the global blob (tables used once per cell, step or
// refactorisation).  Section offsets come from the kernel parameter M.tab.
struct Tabs {
  const unsigned char *base;
  const unsigned char *gbase;
};
template <typename X>
__device__ __forceinline__ const X *tab(const Tabs &tb, int off) {
  return reinterpret_cast<const X *>(tb.base + off);
}
template <typename X>
__device__ __forceinline__ const X *gtab(const Tabs &tb, int off) {
  return reinterpret_cast<const X *>(tb.gbase + off);
}

// Phase bodies that touch only the cell's shared-memory arrays and the tables.

// a2: r_j = k~_j prod y, then f = the f program, from y in Wd[Y]
template <bool STAGED>
__device__ __forceinline__ void f_core(const MechDev &M, const unsigned char *tbase, double *Wd, const int lane) {
  const uint2 *slots = reinterpret_cast<const uint2 *>(tbase + M.tab.rx_slots);
  // two reactions per lane and iteration, so each lane has two products' loads in flight
  const uint32_t wb = smem_addr(Wd), kt = wb + 8u * M.d_KT, rt = wb + 8u * M.d_RT;
  double *const tag = nullptr;
  int j = lane;
#pragma unroll 1
  for (; j + WARP < M.R; j += 2 * WARP) {
    const uint2 s0 = slots[j], s1 = slots[j + WARP];
    double r0 = lds(tag, kt + 8u * j) * lds(tag, wb + (s0.x & 0xffff));
    double r1 = lds(tag, kt + 8u * (j + WARP)) * lds(tag, wb + (s1.x & 0xffff));
    if (M.max_reac > 1) {
      r0 *= lds(tag, wb + (s0.x >> 16));
      r1 *= lds(tag, wb + (s1.x >> 16));
    }
    if (M.max_reac > 2) {
      r0 *= lds(tag, wb + (s0.y & 0xffff));
      r1 *= lds(tag, wb + (s1.y & 0xffff));
    }
    sts(rt + 8u * j, r0);
    sts(rt + 8u * (j + WARP), r1);
  }
  if (j < M.R) {
    const uint2 sl = slots[j];
    double r = lds(tag, kt + 8u * j) * lds(tag, wb + (sl.x & 0xffff));
    if (M.max_reac > 1) r *= lds(tag, wb + (sl.x >> 16));
    if (M.max_reac > 2) r *= lds(tag, wb + (sl.y & 0xffff));
    sts(rt + 8u * j, r);
  }
  __syncwarp();
  run_prog<double, false, STAGED, true, false>(reinterpret_cast<const ushort4 *>(tbase + M.tab.f_ops),
                                               reinterpret_cast<const uint32_t *>(tbase + M.tab.f_runs), M.f_nruns,
                                               M.f_npass, Wd, lane);
}

// a3-a5: M = I - c J(y) in the LU slots from y in Wd[Y], then factor
template <typename T>
__device__ __forceinline__ void mlu_core(const MechDev &M, const unsigned char *tbase, const int prec, double *Wd, T *WL,
                                      const double c, const int lane) {
  for (int i = lane; i < M.m_clear; i += WARP) WL[i] = (T)0;
  __syncwarp();
  unsigned char *wl = reinterpret_cast<unsigned char *>(WL);
  unsigned char *wd = reinterpret_cast<unsigned char *>(Wd);
  const int *diag = reinterpret_cast<const int *>(tbase + M.tab.lu_diag);
  const int *prx = reinterpret_cast<const int *>(tbase + M.tab.pair_rx);
  const unsigned *pother = reinterpret_cast<const unsigned *>(tbase + M.tab.pair_other);
  for (int k = lane; k < M.S; k += WARP) at<T>(wl, diag[k]) = (T)1;
  const double mc = -c;
  // two pairs per lane and iteration (loads in flight together); the pair
  // products go to the slots of the rates, f and f temps, dead while M is formed
  T *const pp = reinterpret_cast<T *>(Wd + M.d_RT);
  const uint32_t wdb = smem_addr(Wd), kt = wdb + 8u * M.d_KT;
  double *const tag = nullptr;
  int pr = lane;
#pragma unroll 1
  for (; pr + WARP < M.n_pairs; pr += 2 * WARP) {
    const int j0 = prx[pr], j1 = prx[pr + WARP];
    const unsigned o0 = pother[pr], o1 = pother[pr + WARP];
    double p0 = mc * lds(tag, kt + 8u * j0), p1 = mc * lds(tag, kt + 8u * j1);
    if (M.max_reac > 1) {
      p0 *= lds(tag, wdb + (o0 & 0xffff));
      p1 *= lds(tag, wdb + (o1 & 0xffff));
    }
    if (M.max_reac > 2) {
      p0 *= lds(tag, wdb + (o0 >> 16));
      p1 *= lds(tag, wdb + (o1 >> 16));
    }
    pp[pr] = (T)p0;
    pp[pr + WARP] = (T)p1;
  }
  if (pr < M.n_pairs) {
    const int j = prx[pr];
    const unsigned o = pother[pr];
    double p = mc * lds(tag, kt + 8u * j);
    if (M.max_reac > 1) p *= lds(tag, wdb + (o & 0xffff));
    if (M.max_reac > 2) p *= lds(tag, wdb + (o >> 16));
    pp[pr] = (T)p;
  }
  __syncwarp();
  // The M program runs on the whole per-cell slice (its operands are the pair
  // products in Wd and the LU slots, constants and temporaries in WL), its ops
  // read from L2 two passes ahead.  The LU program's ops are streamed through a
  // ring in the rates and f slots of Wd, dead once M is formed (too small a
  // region: read from L2 as well).
  run_prog<T, false, false, true, false>(M.m_ops[prec], M.m_runs, M.m_nruns, M.m_npass, reinterpret_cast<T *>(Wd), lane);
  const uint32_t wr = smem_addr(Wd + M.d_RT);            // 8-byte aligned (a double slot)
  if ((M.R + M.S) * 8 >= 8 * 256)
    run_prog_ring<T, false, 8, true, true>(M.lu_ops[prec], M.lu_runs, M.lu_nruns, M.lu_npass, WL, lane, wr);
  else
    run_prog<T, false, false, true, true>(M.lu_ops[prec], M.lu_runs, M.lu_nruns, M.lu_npass, WL, lane);
}

// a5: forward and backward substitution with the LDU factors on the vector in
// WL[X]; it leaves -x there (the programs run without negation).  Staged (the
// persistent driver) the programs are read from shared memory; otherwise they
// are streamed from L2 through a ring in the rates and f slots of Wd, which
// are dead during a solve.  (Streaming them in the staged form too measured
// slower, at 10 cells per SM and at the 11 that it lets fit.)
template <typename T, bool STAGED>
__device__ __forceinline__ void solve_core(const MechDev &M, const unsigned char *tbase, double *Wd, T *WL, const int lane) {
  const ushort4 *fwd = reinterpret_cast<const ushort4 *>(tbase + M.tab.fwd_ops);
  const ushort4 *bwd = reinterpret_cast<const ushort4 *>(tbase + M.tab.bwd_ops);
  T *const W = reinterpret_cast<T *>(Wd);                 // the programs address the whole per-cell slice
  if (STAGED) {
    run_ops<T, false, true>(fwd, M.fwd_npass, W, lane);
    run_ops<T, false, true>(bwd, M.bwd_npass, W, lane);
    return;
  }
  const uint32_t rb = smem_addr(Wd + M.d_RT);            // the rates and f slots: dead during a solve
  const int cap = (M.R + M.S) * 8;
  if (cap >= 8 * 256) {
    run_ops_ring<T, false, 8>(fwd, M.fwd_npass, W, lane, rb);
    run_ops_ring<T, false, 8>(bwd, M.bwd_npass, W, lane, rb);
  } else if (cap >= 4 * 256) {
    run_ops_ring<T, false, 4>(fwd, M.fwd_npass, W, lane, rb);
    run_ops_ring<T, false, 4>(bwd, M.bwd_npass, W, lane, rb);
  } else {
    run_ops<T, false, false>(fwd, M.fwd_npass, W, lane);
    run_ops<T, false, false>(bwd, M.bwd_npass, W, lane);
  }
}

template <typename T, int KS, bool STAGED>
struct Cell {
  const MechDev &M;
  const SolveParams &P;
  const Tabs &tb;
  double *Wd;
  T *WL;
  int lane;
  int pos[KS];        // pivot position of this lane's species
  bool own[KS];       // species index < S
  double invS;        // 1 / number of species (norm weight)

  __device__ __forceinline__ Cell(const MechDev &m, const SolveParams &p, const Tabs &t, double *wd, T *wl, int l)
      : M(m), P(p), tb(t), Wd(wd), WL(wl), lane(l) {
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      const int s = lane + WARP * k;
      own[k] = s < M.S;
      pos[k] = own[k] ? __ldg(M.sp_pos + s) : 0;
    }
    invS = 1.0 / (double)M.S;
  }

  __device__ __forceinline__ void init_constants() {
    unsigned char *wd = reinterpret_cast<unsigned char *>(Wd);
    unsigned char *wl = reinterpret_cast<unsigned char *>(WL);
    for (int k = lane; k < M.d_nconst; k += WARP) at<double>(wd, gtab<int>(tb, M.tab.dconst_off)[k]) = gtab<double>(tb, M.tab.dconst_val)[k];
    for (int k = lane; k < M.L_nconst; k += WARP) at<T>(wl, gtab<int>(tb, M.tab.Lconst_off)[k]) = (T)gtab<double>(tb, M.tab.Lconst_val)[k];
  }

  // warp sum of (v_i w_i)^2 over this cell's species
  __device__ __forceinline__ double sumsq(const double (&v)[KS], const double (&w)[KS]) const {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < KS; ++k)
      if (own[k]) {
        const double t = v[k] * w[k];
        s = fma(t, t, s);
      }
    return warp_sum_nn(s);
  }

  __device__ __forceinline__ void weights(const double (&y)[KS], double (&w)[KS]) const {
#pragma unroll
    for (int k = 0; k < KS; ++k) w[k] = own[k] ? recip_nr(fma(P.rtol, fabs(y[k]), P.atol)) : 0.0;
  }

  // a2: f(y) into registers
  __device__ __forceinline__ void eval_f(const double (&y)[KS], double (&f)[KS]) {
#pragma unroll
    for (int k = 0; k < KS; ++k)
      if (own[k]) Wd[M.d_Y + lane + WARP * k] = y[k];
    __syncwarp();
    f_core<STAGED>(M, tb.base, Wd, lane);
#pragma unroll
    for (int k = 0; k < KS; ++k) f[k] = own[k] ? Wd[M.d_F + lane + WARP * k] : 0.0;
    __syncwarp();
  }

  // a3-a5: M = I - c J(y) in the LU slots, then factor
  __device__ __forceinline__ void form_and_factor(double c, const double (&y)[KS]) {
#pragma unroll
    for (int k = 0; k < KS; ++k)
      if (own[k]) Wd[M.d_Y + lane + WARP * k] = y[k];
    mlu_core<T>(M, tb.base, P.prec, Wd, WL, c, lane);
  }

  // a5: x = M^{-1} b with the factored M
  __device__ __forceinline__ void solve(const double (&b)[KS], double (&x)[KS]) {
#pragma unroll
    for (int k = 0; k < KS; ++k)
      if (own[k]) reinterpret_cast<T *>(Wd + M.d_Y)[pos[k]] = (T)b[k];   // the solve vector: y's slots
    __syncwarp();
    solve_core<T, STAGED>(M, tb.base, Wd, WL, lane);
#pragma unroll
    for (int k = 0; k < KS; ++k) x[k] = own[k] ? -(double)reinterpret_cast<const T *>(Wd + M.d_Y)[pos[k]] : 0.0;
    __syncwarp();
  }
};

// History rescale for a step ratio eta at order q: D'_i = sum_{m>=i} T_im(eta) D_m,
// T_im a polynomial in eta whose coefficients the host precomputed.
template <int KS>
__device__ __forceinline__ void rescale(double (&D)[NROW][KS], int q, double eta, const double *coef, int lane) {
  // lane (i-1)*QMAX + (m-1) evaluates T_im
  double tv = 0.0;
  if (lane < QMAX * QMAX) {
    const double *cp = coef + lane * (QMAX + 1);
    tv = __ldg(cp + QMAX);
#pragma unroll
    for (int p = QMAX - 1; p >= 0; --p) tv = fma(tv, eta, __ldg(cp + p));
  }
  // in place, rows ascending: row i reads only rows m >= i, still unchanged
#pragma unroll
  for (int i = 1; i <= QMAX; ++i) {
    if (i > q) break;
    double nd[KS];
#pragma unroll
    for (int k = 0; k < KS; ++k) nd[k] = 0.0;
#pragma unroll
    for (int mm = 1; mm <= QMAX; ++mm) {
      if (mm > q) break;
      if (mm < i) continue;
      const double t = __shfl_sync(FULL, tv, (i - 1) * QMAX + (mm - 1));
#pragma unroll
      for (int k = 0; k < KS; ++k) nd[k] = fma(t, D[mm][k], nd[k]);
    }
#pragma unroll
    for (int k = 0; k < KS; ++k) D[i][k] = nd[k];
  }
}

// Row access with a runtime row index.  Written as a switch with constant
// row numbers: a loop of "if (m == r)" selects gets canonicalised into a
// dynamically indexed access, which moves the whole history into local memory.
template <int KS>
__device__ __forceinline__ void get_row(const double (&D)[NROW][KS], int r, double (&out)[KS]) {
#define CHEM_ROW_CASE(R_)                                 \
  case R_:                                               \
    _Pragma("unroll") for (int k = 0; k < KS; ++k) out[k] = D[R_][k]; \
    break;
  switch (r) {
    CHEM_ROW_CASE(0) CHEM_ROW_CASE(1) CHEM_ROW_CASE(2) CHEM_ROW_CASE(3)
    CHEM_ROW_CASE(4) CHEM_ROW_CASE(5) CHEM_ROW_CASE(6) CHEM_ROW_CASE(7)
    default:
      _Pragma("unroll") for (int k = 0; k < KS; ++k) out[k] = 0.0;
  }
#undef CHEM_ROW_CASE
}

// Accepted step at order q: D_{q+2} = d - D_{q+1}, D_{q+1} = d, then
// D_m += D_{m+1} for m = q .. 0.
template <int KS>
__device__ __forceinline__ void accept_update(double (&D)[NROW][KS], int q, const double (&d)[KS]) {
#define CHEM_UPD_CASE(Q_)                                                      \
  case Q_:                                                                    \
    _Pragma("unroll") for (int k = 0; k < KS; ++k) {                          \
      D[Q_ + 2][k] = d[k] - D[Q_ + 1][k];                                     \
      D[Q_ + 1][k] = d[k];                                                    \
    }                                                                         \
    _Pragma("unroll") for (int m = Q_; m >= 0; --m)                           \
      _Pragma("unroll") for (int k = 0; k < KS; ++k) D[m][k] += D[m + 1][k];  \
    break;
  switch (q) {
    CHEM_UPD_CASE(1) CHEM_UPD_CASE(2) CHEM_UPD_CASE(3) CHEM_UPD_CASE(4) CHEM_UPD_CASE(5)
    default:
      break;
  }
#undef CHEM_UPD_CASE
}

// Inputs of one cell: y0 into registers, a1 rate constants into Wd[KT].
// Returns true (warp-uniform) if any input or rate constant is not finite or
// T, P are not positive.
template <int KS>
__device__ __forceinline__ bool load_cell(const MechDev &M, const CellsDev &C, double *Wd, const int lane, const int64_t cell,
                          const bool (&own)[KS], double (&y0)[KS]) {
  const int64_t NC = C.n_cells;
  const int R = M.R;
  const double Tc = C.T[cell], Pc = C.P[cell];
  bool bad = !(Tc > 0.0) || !(Pc > 0.0) || !isfinite(Tc) || !isfinite(Pc);
#pragma unroll
  for (int k = 0; k < KS; ++k) {
    y0[k] = own[k] ? C.y[(int64_t)(lane + WARP * k) * NC + cell] : 0.0;
    if (own[k] && !isfinite(y0[k])) bad = true;
  }
  if (!__any_sync(FULL, bad)) {
    const double n_air = air_number_density(Tc, Pc);
    for (int j = lane; j < R; j += WARP) {
      const double kj = rate_constant(M, C, j, cell, Tc, n_air);
      Wd[M.d_KT + j] = kj;
      if (!isfinite(kj)) bad = true;
    }
  }
  bad = __any_sync(FULL, bad);
  __syncwarp();
  return bad;
}

// Reductions across the warps of a coupled group (the paper's multi-cell
// system: one integration over a group of cells, one warp per cell; a block
// holds several groups, each with its own named barrier).  Each warp's partial
// goes to a shared slot; after the group's barrier every thread combines the
// slots in warp order, so all warps of the group see the same bits and take
// the same decisions.  Uncoupled: identity.
template <bool COUPLED>
struct Grp {
  double *slot;     // [g] in shared memory, this group's
  int w, g, bar;    // warp index in the group, warps in the group, named barrier of the group
  __device__ __forceinline__ void sync() const {
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(g * WARP) : "memory");
  }
  __device__ __forceinline__ double sum(double v) const {
    if (!COUPLED) return v;
    sync();                              // earlier readers of the slots are done
    if ((threadIdx.x & (WARP - 1)) == 0) slot[w] = v;
    sync();
    double s = 0.0;
    for (int i = 0; i < g; ++i) s += slot[i];
    return s;
  }
  __device__ __forceinline__ double min(double v) const {
    if (!COUPLED) return v;
    sync();
    if ((threadIdx.x & (WARP - 1)) == 0) slot[w] = v;
    sync();
    double s = slot[0];
    for (int i = 1; i < g; ++i) s = fmin(s, slot[i]);
    return s;
  }
  __device__ __forceinline__ bool any(bool b) const { return COUPLED ? sum(b ? 1.0 : 0.0) > 0.0 : b; }
};

// Event tape of one cell for the discrete adjoint (event kinds and rows as
// CellsDev documents them).  Every lane keeps the counters; lane 0 writes the
// events, each lane its own species of a row.  With ON false every method is
// empty and the solve kernel carries no recording state.
template <int KS, bool ON>
struct Recorder {
  const CellsDev &C;
  int64_t cell;
  double *yrows;        // this cell's rows
  int n, rows, S;
  bool on, over;   // on == ON
  __device__ __forceinline__ Recorder(const CellsDev &c, int64_t cl, int s)
      : C(c), cell(cl), yrows(nullptr), n(0), rows(0), S(s), on(ON), over(false) {
    if (ON) {
      n = C.tape_n[cell];
      rows = C.tape_rows[cell];
      yrows = C.ytape + cell * (int64_t)C.row_cap * s;
    }
  }
  __device__ __forceinline__ void event(int kind, int q, double val, int lane) {
    if (lane == 0) {
      const int64_t i = cell * (int64_t)C.tape_cap + n;
      C.tape_kq[i] = kind | (q << 8);
      C.tape_val[i] = val;
    }
    n++;
  }
  __device__ __forceinline__ void write_row(int r, const double (&y)[KS], int lane) {
#pragma unroll
    for (int k = 0; k < KS; ++k)
      if (lane + WARP * k < S) yrows[(int64_t)r * S + lane + WARP * k] = y[k];
  }
  // an event without a row (RESCALE, STEP, PROJECT)
  __device__ __forceinline__ void push(int kind, int q, double val, int lane) {
    if (!ON) return;
    if (n >= C.tape_cap) {
      over = true;
      return;
    }
    event(kind, q, val, lane);
  }
  // an event with a row (INIT, REFACTOR); a REFACTOR's q is its row index
  __device__ __forceinline__ void push_row(int kind, int q, double val, const double (&y)[KS], int lane) {
    if (!ON) return;
    if (n >= C.tape_cap || rows >= C.row_cap) {
      over = true;
      return;
    }
    write_row(rows, y, lane);
    event(kind, kind == EV_REFACTOR ? rows : q, val, lane);
    rows++;
  }
  // iterate it of the current attempt, kept only if the step is accepted
  __device__ __forceinline__ void iterate(int it, const double (&y)[KS], int lane) {
    if (ON && rows + it < C.row_cap) write_row(rows + it, y, lane);
  }
  // acceptance: the attempt's K iterates become ITER events
  __device__ __forceinline__ void accept_iters(int K, int lane) {
    if (!ON) return;
    if (n + K > C.tape_cap || rows + K > C.row_cap) {
      over = true;
      return;
    }
    for (int k = 0; k < K; ++k) event(EV_ITER, k, 0.0, lane);
    rows += K;
  }
  // acceptance: the species the attempt projected onto y = 0, ascending
  __device__ __forceinline__ void accept_projections(const unsigned (&pm)[KS], int lane) {
    if (!ON) return;
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      unsigned b = pm[k];
      while (b) {
        const int l = __ffs(b) - 1;
        b &= b - 1;
        push(EV_PROJECT, l + WARP * k, 0.0, lane);
      }
    }
  }
  __device__ __forceinline__ void finish(bool failed, int lane) {
    if (!ON || lane != 0) return;
    C.tape_n[cell] = n;
    C.tape_rows[cell] = rows;
    if (over || failed) C.tape_bad[cell] = 1;
  }
};

// One cell (COUPLED: one cell of a coupled group; cell < 0 marks a warp
// without a cell in a ragged last group, which follows the group's control
// flow and contributes nothing).  invN scales the norms' sums: 1/S alone,
// 1/(cells in the group * S) coupled.  The controller's tests compare the
// raw sums sum (v_i w_i)^2 with bounds the host multiplied by S (tables thr2,
// thr3, lim); coupled, the group's sums are first scaled by gsc = 1/(cells
// in the group).
template <typename T, int KS, bool STAGED, bool REC, bool COUPLED>
__device__ __forceinline__ void solve_cell(const MechDev &M, const CellsDev &C, const SolveParams &P, const Tabs &tb, double *Wd,
                           T *WL, const int lane, const int64_t cell, const Grp<COUPLED> &grp, const double invN,
                           const double gsc) {
  const int64_t NC = C.n_cells;
  chem_cell_stats st = {};
  int status = CHEM_CELL_OK;
  const bool phantom = COUPLED && cell < 0;

  Cell<T, KS, STAGED> cl(M, P, tb, Wd, WL, lane);
  if (phantom) {
#pragma unroll
    for (int k = 0; k < KS; ++k) cl.own[k] = false;
  }
  cl.init_constants();
  double y0[KS];
#pragma unroll
  for (int k = 0; k < KS; ++k) y0[k] = 0.0;
  const bool bad = grp.any(phantom ? false : load_cell<KS>(M, C, Wd, lane, cell, cl.own, y0));
  Recorder<KS, REC> rec(C, cell, M.S);

  const double dt = P.dt;
  int q = 1;
  double h = 0.0;
  double D[NROW][KS];
  if (bad) {
    status = CHEM_CELL_BAD_INPUT;
  } else {
    double w[KS], f[KS], tmp[KS], f0[KS];
    cl.weights(y0, w);
    // initial step (order 1)
    cl.eval_f(y0, f0);
    st.f_evals++;
    const double d0 = sqrt(grp.sum(cl.sumsq(y0, w)) * invN), d1 = sqrt(grp.sum(cl.sumsq(f0, w)) * invN);
    double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 * dt : 0.01 * d0 / d1;
    if (h0 > dt) h0 = dt;
#pragma unroll
    for (int k = 0; k < KS; ++k) tmp[k] = y0[k] + h0 * f0[k];
    cl.eval_f(tmp, f);
    st.f_evals++;
#pragma unroll
    for (int k = 0; k < KS; ++k) tmp[k] = f[k] - f0[k];
    const double d2 = sqrt(grp.sum(cl.sumsq(tmp, w)) * invN) / h0;
    const double dm = d1 > d2 ? d1 : d2;
    const double h1 = (dm <= 1e-15) ? fmax(1e-6 * dt, h0 * 1e-3) : sqrt(0.01 / dm);
    h = fmin(fmin(100.0 * h0, h1), dt);
#pragma unroll
    for (int m = 0; m < NROW; ++m)
#pragma unroll
      for (int k = 0; k < KS; ++k) D[m][k] = 0.0;
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      D[0][k] = y0[k];
      D[1][k] = h * f0[k];
    }
    rec.push_row(EV_INIT, q, h, y0, lane);

    double t = 0.0, cM = 0.0, icM = 0.0, rho2 = 1.0;   // rho2: squared convergence-rate estimate
    int n_eq = 0, have_M = 0, force_M = 0, n_since_M = 0, nef = 0, ncf = 0, last = 0;
    const int qmax = P.max_order;
    double ypred[KS], psi[KS], d[KS], y[KS], x[KS];

    const double *thr2 = gtab<double>(tb, M.tab.thr2), *thr3 = gtab<double>(tb, M.tab.thr3);
    const double *gfac = gtab<double>(tb, M.tab.g), *lim = gtab<double>(tb, M.tab.lim);
    for (;;) {
      if (st.steps >= P.max_steps) { status = CHEM_CELL_MAX_STEPS; break; }
      // dt - t >= +0 always (t < dt inside the loop)
      if (le_nn(dt - t, h * (1.0 + STRETCH))) {
        const double hn = dt - t;
        if (!eq_fp(hn, h)) {
          rescale<KS>(D, q, hn / h, M.rescale_coef, lane);
          rec.push(EV_RESCALE, q, hn / h, lane);
          h = hn;
          n_eq = 0;
        }
        last = 1;
      } else {
        last = 0;
      }
      if (!last && eq_fp(t + h, t)) { status = CHEM_CELL_H_TOO_SMALL; break; }

      const double iq = c_igam[q];
      const double c = h * iq;
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        ypred[k] = D[0][k];
        psi[k] = 0.0;
      }
#pragma unroll
      for (int m = 1; m <= QMAX; ++m) {
        if (m > q) break;
        const double gm = c_gam[m];
#pragma unroll
        for (int k = 0; k < KS; ++k) {
          ypred[k] += D[m][k];
          psi[k] = fma(gm, D[m][k], psi[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < KS; ++k) psi[k] *= iq;

      int fresh = 0;
      if (!have_M || force_M || gt_nn(__longlong_as_double(__double_as_longlong(fma(c, icM, -1.0)) & ABS_MASK), DGMAX) ||
          n_since_M >= MSBP) {
        cl.form_and_factor(c, ypred);
        have_M = 1;
        cM = c;
        icM = recip_nr(c);
        n_since_M = 0;
        rho2 = 1.0;
        fresh = 1;
        st.jac_evals++;
        rec.push_row(EV_REFACTOR, 0, c, ypred, lane);
      }
      force_M = 0;
      const bool scaled = !eq_fp(c, cM);
      double scale = 1.0;
      if (scaled) scale = 2.0 * recip_nr(fma(c, icM, 1.0));
      const double tol2 = lim[8 + q];     // S (0.1 (q+1))^2

#pragma unroll
      for (int k = 0; k < KS; ++k) {
        d[k] = 0.0;
        y[k] = ypred[k];
      }
      double del2 = 0.0, del2_prev = 0.0, idel2_prev = 0.0;   // idel2_prev = 1 / del2_prev
      int conv = 0;
      int n_it = 0;
      for (int it = 0; it < NEWTON_MAXITER; ++it) {
        rec.iterate(it, y, lane);
        n_it = it + 1;
        cl.eval_f(y, f);
        st.f_evals++;
#pragma unroll
        for (int k = 0; k < KS; ++k) tmp[k] = c * f[k] - psi[k] - d[k];
        cl.solve(tmp, x);
        st.solves++;
        if (scaled) {
#pragma unroll
          for (int k = 0; k < KS; ++k) x[k] *= scale;
        }
        del2 = grp.sum(cl.sumsq(x, w));
        if (COUPLED) del2 *= gsc;
#pragma unroll
        for (int k = 0; k < KS; ++k) {
          d[k] += x[k];
          y[k] = ypred[k] + d[k];
        }
        st.newton_iters++;
        if (it > 0) rho2 = max_nn(CRDOWN * CRDOWN * rho2, del2 * idel2_prev);
        if (le_nn(le_nn(rho2, 1.0) ? del2 * rho2 : del2, tol2)) { conv = 1; break; }
        if (it > 0 && gt_nn(del2, RDIV * RDIV * del2_prev)) break;
        // not converged, so del2 > tol2 >= 1e-2 S (q >= 1): a normal number
        del2_prev = del2;
        idel2_prev = recip_nr(del2);
      }
      if (!conv) {
        st.conv_fails++;
        ncf++;
        if (ncf >= MXNCF) { status = CHEM_CELL_CONV_FAIL; break; }
        if (!fresh) {
          force_M = 1;
        } else {
          rescale<KS>(D, q, ETA_CF, M.rescale_coef, lane);
          rec.push(EV_RESCALE, q, ETA_CF, lane);
          h *= ETA_CF;
          n_eq = 0;
        }
        continue;
      }

      // inequality constraint y >= 0
      unsigned pm[KS];          // species projected onto y = 0 (ballot per register slot)
#pragma unroll
      for (int k = 0; k < KS; ++k) pm[k] = 0u;
      {
        bool neg = false;
#pragma unroll
        for (int k = 0; k < KS; ++k) neg |= cl.own[k] && lt0(y[k]);
        if (grp.any(__any_sync(FULL, neg))) {
          double vs = 0.0, eta_c = 1.0;
#pragma unroll
          for (int k = 0; k < KS; ++k)
            if (cl.own[k] && lt0(y[k])) {
              const double v = y[k] * w[k];
              vs = fma(v, v, vs);
              const double r = (D[0][k] > 0.0) ? D[0][k] / (D[0][k] - y[k]) : 0.0;
              eta_c = fmin(eta_c, r);
            }
          vs = grp.sum(warp_sum_nn(vs));
          if (COUPLED) vs *= gsc;
          eta_c = grp.min(warp_min(eta_c));
          if (le_nn(vs, tol2)) {
#pragma unroll
            for (int k = 0; k < KS; ++k) {
              const bool p = cl.own[k] && lt0(y[k]);
              if (p) {
                d[k] -= y[k];
                y[k] = 0.0;
              }
              if (REC) pm[k] = __ballot_sync(FULL, p);
            }
          } else {
            st.rejects++;
            nef++;
            if (nef >= MXNEF) { status = CHEM_CELL_ERR_FAIL; break; }
            double eta = ETA_CST_SAFETY * eta_c;
            if (eta < ETA_CST_MIN) eta = ETA_CST_MIN;
            rescale<KS>(D, q, eta, M.rescale_coef, lane);
            rec.push(EV_RESCALE, q, eta, lane);
            h *= eta;
            n_eq = 0;
            continue;
          }
        }
      }

      // local error test: (||d|| / (q+1))^2 <= 1, as the raw sum against S (q+1)^2
      double err2 = grp.sum(cl.sumsq(d, w));
      if (COUPLED) err2 *= gsc;
      const int ie = grid_idx(thr2, err2, q, lane);
      if (!le_nn(err2, lim[q])) {
        st.rejects++;
        nef++;
        if (nef >= MXNEF) { status = CHEM_CELL_ERR_FAIL; break; }
        double eta = gfac[ie];
        if (nef >= 2 && gt_nn(eta, ETA_MXF)) eta = ETA_MXF;
        if (nef >= 3 && q > 1) q -= 1;
        rescale<KS>(D, q, eta, M.rescale_coef, lane);
        rec.push(EV_RESCALE, q, eta, lane);
        h *= eta;
        n_eq = 0;
        continue;
      }

      // accept: update the backward differences
      t = last ? dt : t + h;
      st.steps++;
      st.order_sum += q;
      n_since_M++;
      nef = 0;
      ncf = 0;
      accept_update<KS>(D, q, d);
      rec.accept_iters(n_it, lane);
      rec.accept_projections(pm, lane);
      rec.push(EV_STEP, q, c, lane);
      if (last) break;
      n_eq++;

      // next factor: grid indices compare as the factors do (g_i increasing)
      int ieta = ie;
      int qn = q;
      if (n_eq >= q + 1) {
        if (q > 1) {
          double row[KS];
          get_row<KS>(D, q, row);
          double e2 = grp.sum(cl.sumsq(row, w));       // (||D_q|| / q)^2 against row q-1
          if (COUPLED) e2 *= gsc;
          const int im = grid_idx(thr2, e2, q - 1, lane);
          if (im > ieta) { ieta = im; qn = q - 1; }
        }
        if (q < qmax) {
          double row[KS];
          get_row<KS>(D, q + 2, row);
          double e2 = grp.sum(cl.sumsq(row, w));       // (||D_{q+2}|| / (q+2))^2 against row q+1
          if (COUPLED) e2 *= gsc;
          const int ip = grid_idx(thr3, e2, q + 1, lane);
          if (ip > ieta) { ieta = ip; qn = q + 1; }
        }
      }
      const double eta = gfac[ieta];
      if (le_nn(THRESH, eta)) {
        q = qn;
        rescale<KS>(D, q, eta, M.rescale_coef, lane);
        rec.push(EV_RESCALE, q, eta, lane);
        h *= eta;
        n_eq = 0;
      }
      double y_acc[KS];
#pragma unroll
      for (int k = 0; k < KS; ++k) y_acc[k] = D[0][k];
      cl.weights(y_acc, w);
    }
    if (status == CHEM_CELL_OK) {
      bool nf = false;
#pragma unroll
      for (int k = 0; k < KS; ++k) nf |= cl.own[k] && !isfinite(D[0][k]);
      if (grp.any(__any_sync(FULL, nf))) status = CHEM_CELL_NONFINITE;
    }
    if (status == CHEM_CELL_OK) {
#pragma unroll
      for (int k = 0; k < KS; ++k)
        if (cl.own[k]) C.y[(int64_t)(lane + WARP * k) * NC + cell] = D[0][k];
    }
  }
  rec.finish(status != CHEM_CELL_OK, lane);
  if (lane == 0 && !phantom) {
    st.status = status;
    st.final_order = q;
    st.final_h = h;
    C.stats[cell] = st;
  }
  __syncwarp();
}

// Stage the table blob into the first `bytes` of shared memory with one TMA
// bulk copy.  The wait is bounded (`limit` polls of the barrier); if it runs
// out, the block counts the event in stage[0] and copies the blob with
// ordinary loads instead.  A late bulk copy then writes the same bytes to the
// same place, so whichever lands last leaves the tables intact; the block
// waits (bounded again) for that copy before it exits.  Keeping the tables in
// shared memory on both paths lets every table read use shared-memory loads.
__device__ bool stage_tables(const unsigned char *blob, int bytes, unsigned char *smem, uint64_t *bar,
                             unsigned long long *stage, long long limit) {
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, (uint32_t)bytes);
    tma_load_1d(smem, blob, (uint32_t)bytes, bar);
  }
  const bool ok = __syncthreads_and(mbar_wait(bar, 0, limit));
  if (!ok) {
    const uint4 *src = reinterpret_cast<const uint4 *>(blob);
    uint4 *dst = reinterpret_cast<uint4 *>(smem);
    for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    __syncthreads();
    if (threadIdx.x == 0 && stage) atomicAdd(stage, 1ull);
  }
  return ok;
}

template <typename T, int KS, bool STAGED, bool REC, bool COUPLED>
__global__ void __launch_bounds__(MAX_WARPS_PER_BLOCK * WARP) solve_kernel(const __grid_constant__ MechDev M, const CellsDev C, const SolveParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t tma_bar;
  __shared__ double grp_slot[COUPLED ? MAX_WARPS_PER_BLOCK : 1];
  __shared__ long long grp_next[COUPLED ? MAX_WARPS_PER_BLOCK : 1];
  const int lane = threadIdx.x & (WARP - 1);
  const int warp = threadIdx.x / WARP;
  Tabs tb;
  tb.gbase = M.blob[P.prec];
  bool staged_ok = true;
  if (STAGED) {
    staged_ok = stage_tables(M.blob[P.prec], P.tab_bytes, smem, &tma_bar, C.stage, P.stage_wait);
    tb.base = smem;
  } else {
    tb.base = M.blob[P.prec];
  }
  double *Wd = reinterpret_cast<double *>(smem + P.tab_bytes + (size_t)warp * P.cell_bytes);
  T *WL = reinterpret_cast<T *>(Wd + P.wd_pad);
  Grp<COUPLED> grp;
  const double invS = 1.0 / (double)M.S;
  if (COUPLED) {
    // groups of P.couple consecutive cells, P.warps_per_block / P.couple per
    // block, each with named barrier 1 + its index; with the queue, groups are
    // handed out whole
    const int G = P.couple, gpb = P.warps_per_block / G, gl = warp / G;
    grp.slot = grp_slot + gl * G;
    grp.w = warp - gl * G;
    grp.g = G;
    grp.bar = 1 + gl;
    if (gl < gpb) {
      for (int64_t gi = (int64_t)blockIdx.x * gpb + gl;;) {
        if (C.queue) {
          grp.sync();
          if (grp.w == 0 && lane == 0) grp_next[gl] = (long long)atomicAdd(C.queue, 1ull);
          grp.sync();
          gi = grp_next[gl];
          if (C.order && gi * G < C.n_cells) gi = __ldg(C.order + gi);   // groups most expensive first
        }
        const int64_t c0 = gi * G;
        if (c0 >= C.n_cells) break;
        const int n_act = (int)((C.n_cells - c0) < G ? (C.n_cells - c0) : G);
        const int64_t cell = grp.w < n_act ? c0 + grp.w : -1;
        solve_cell<T, KS, STAGED, REC, COUPLED>(M, C, P, tb, Wd, WL, lane, cell, grp, 1.0 / (double)(n_act * M.S),
                                                1.0 / (double)n_act);
        if (!C.queue) break;
      }
    }
  } else if (C.queue) {
    for (;;) {
      long long cell = 0;
      if (lane == 0) cell = (long long)atomicAdd(C.queue, 1ull);
      cell = __shfl_sync(FULL, cell, 0);
      if (cell >= C.n_cells) break;
      if (C.order) cell = __ldg(C.order + cell);
      solve_cell<T, KS, STAGED, REC, COUPLED>(M, C, P, tb, Wd, WL, lane, cell, grp, invS, 1.0);
    }
  } else {
    const int64_t cell = (int64_t)blockIdx.x * P.warps_per_block + warp;
    if (cell < C.n_cells) solve_cell<T, KS, STAGED, REC, COUPLED>(M, C, P, tb, Wd, WL, lane, cell, grp, invS, 1.0);
  }
  // a late bulk copy must land before the block exits (its shared memory is
  // then handed to another block); one thread waits, bounded, and counts a
  // wait that ran out in stage[1]
  if (STAGED && !staged_ok && threadIdx.x == 0) {
    if (!mbar_wait(&tma_bar, 0, STAGE_WAIT_DEFAULT) && C.stage) atomicAdd(C.stage + 1, 1ull);
  }
}

// Diagnostic: per cell, f(y) (mode 0) or x = (I - c J(y))^{-1} b (mode 1),
// using the same device routines as the solve.
template <typename T, int KS>
__global__ void __launch_bounds__(MAX_WARPS_PER_BLOCK * WARP) probe_kernel(const __grid_constant__ MechDev M, const CellsDev C, const SolveParams P,
                                                                  int mode, double c, const double *yin, const double *bin,
                                                                  double *out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & (WARP - 1);
  const int warp = threadIdx.x / WARP;
  const int64_t cell = (int64_t)blockIdx.x * P.warps_per_block + warp;
  if (cell >= C.n_cells) return;
  Tabs tb;
  tb.base = tb.gbase = M.blob[P.prec];
  double *Wd = reinterpret_cast<double *>(smem + (size_t)warp * P.cell_bytes);
  T *WL = reinterpret_cast<T *>(Wd + P.wd_pad);
  Cell<T, KS, false> cl(M, P, tb, Wd, WL, lane);
  cl.init_constants();
  double y0[KS];
  load_cell<KS>(M, C, Wd, lane, cell, cl.own, y0);
  const int64_t NC = C.n_cells;
  double y[KS], b[KS], r[KS];
#pragma unroll
  for (int k = 0; k < KS; ++k) {
    const int64_t i = (int64_t)(lane + WARP * k) * NC + cell;
    y[k] = cl.own[k] ? yin[i] : 0.0;
    b[k] = (cl.own[k] && bin) ? bin[i] : 0.0;
  }
  if (mode == 0) {
    cl.eval_f(y, r);
  } else {
    cl.form_and_factor(c, y);
    cl.solve(b, r);
  }
#pragma unroll
  for (int k = 0; k < KS; ++k)
    if (cl.own[k]) out[(int64_t)(lane + WARP * k) * NC + cell] = r[k];
}

// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum,
// once per device and kernel: a host call at every launch would sit between
// the launches on the timeline.
template <auto Kernel>
cudaError_t allow_max_smem() {
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && done[dev]) return cudaSuccess;
  int optin = 0;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, Kernel)) != cudaSuccess) return e;
  e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess && dev < 64) done[dev] = true;
  return e;
}

template <typename T, int KS>
cudaError_t launch_probe_t(const MechDev &M, const CellsDev &C, const SolveParams &P, int mode, double c,
                           const double *y, const double *b, double *out, cudaStream_t stream) {
  const size_t smem = (size_t)P.cell_bytes * P.warps_per_block;
  cudaError_t e = allow_max_smem<probe_kernel<T, KS>>();
  if (e != cudaSuccess) return e;
  const int blocks = (int)((C.n_cells + P.warps_per_block - 1) / P.warps_per_block);
  probe_kernel<T, KS><<<blocks, P.warps_per_block * WARP, smem, stream>>>(M, C, P, mode, c, y, b, out);
  return cudaGetLastError();
}

template <typename T, int KS, bool STAGED, bool REC, bool COUPLED>
cudaError_t configure_t() {
  static bool configured[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && configured[dev]) return cudaSuccess;
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, solve_kernel<T, KS, STAGED, REC, COUPLED>);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(solve_kernel<T, KS, STAGED, REC, COUPLED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess && dev < 64) configured[dev] = true;
  return e;
}

template <typename T, int KS, bool STAGED>
int occupancy_t(int warps_per_block, size_t smem) {
  if (configure_t<T, KS, STAGED, false, false>() != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, solve_kernel<T, KS, STAGED, false, false>, warps_per_block * WARP,
                                                    smem) != cudaSuccess)
    return 0;
  return n;
}

template <typename T, int KS, bool STAGED, bool REC, bool COUPLED>
cudaError_t launch_rec_t(const MechDev &M, const CellsDev &C, const SolveParams &P, int blocks, cudaStream_t stream) {
  const size_t smem = P.smem_bytes > 0 ? (size_t)P.smem_bytes : (size_t)P.tab_bytes + (size_t)P.cell_bytes * P.warps_per_block;
  cudaError_t e = configure_t<T, KS, STAGED, REC, COUPLED>();
  if (e != cudaSuccess) return e;
  solve_kernel<T, KS, STAGED, REC, COUPLED><<<blocks, P.warps_per_block * WARP, smem, stream>>>(M, C, P);
  return cudaGetLastError();
}

// The recording kernel and the coupled (multi-cell) kernel exist for the
// FP64 iteration only; they do not combine.
template <typename T, int KS, bool STAGED>
cudaError_t launch_t(const MechDev &M, const CellsDev &C, const SolveParams &P, int blocks, bool coupled,
                     cudaStream_t stream) {
  if constexpr (std::is_same<T, double>::value) {
    if (C.tape_n && coupled) return cudaErrorInvalidValue;
    if (C.tape_n) return launch_rec_t<T, KS, STAGED, true, false>(M, C, P, blocks, stream);
    if (coupled) return launch_rec_t<T, KS, STAGED, false, true>(M, C, P, blocks, stream);
  } else {
    if (C.tape_n || coupled) return cudaErrorInvalidValue;
  }
  return launch_rec_t<T, KS, STAGED, false, false>(M, C, P, blocks, stream);
}

template <typename T, bool STAGED>
int occupancy_ks(const MechDev &M, int warps_per_block, size_t smem) {
  switch ((M.S + WARP - 1) / WARP) {
    case 1: return occupancy_t<T, 1, STAGED>(warps_per_block, smem);
    case 2: return occupancy_t<T, 2, STAGED>(warps_per_block, smem);
    case 3: return occupancy_t<T, 3, STAGED>(warps_per_block, smem);
    case 4: return occupancy_t<T, 4, STAGED>(warps_per_block, smem);
    default: return 0;
  }
}

template <typename T, bool STAGED>
cudaError_t launch_ks(const MechDev &M, const CellsDev &C, const SolveParams &P, int blocks, bool coupled,
                      cudaStream_t stream) {
  switch ((M.S + WARP - 1) / WARP) {
    case 1: return launch_t<T, 1, STAGED>(M, C, P, blocks, coupled, stream);
    case 2: return launch_t<T, 2, STAGED>(M, C, P, blocks, coupled, stream);
    case 3: return launch_t<T, 3, STAGED>(M, C, P, blocks, coupled, stream);
    case 4: return launch_t<T, 4, STAGED>(M, C, P, blocks, coupled, stream);
    default: return cudaErrorInvalidValue;
  }
}


// ============================================================== discrete adjoint
// The exact adjoint of the forward solve with its controls frozen (Background:
// CVODE's BDF/Newton integration is the map being differentiated).  The
// forward records, per cell, every operation on the BDF history and the
// states the corrector evaluated f and J at (REFACTOR and ITER rows), so the
// backward needs no re-solve: one warp per cell walks the tape in reverse
// carrying the adjoints lambda of the history rows D_0..D_7 in registers.
//   STEP      lambda_d from the history update; projected species pass
//             their lambda_d to lambda_ypred with a minus sign;
//   ITER k    g = s M^{-T} lambda_d (the LU of the REFACTOR in force, then
//             U^T and L^T solves), J(y_k)^T g and nu_j . g by pass programs
//             on the extended Wd array: lambda_d += c J^T g - g,
//             lambda_ypred += c J^T g, lambda_psi -= g,
//             dL/dtheta_j += c r_j(y_k) (nu_j . g); after k = 0 lambda_ypred
//             and lambda_psi fold into lambda_0..q;
//   RESCALE   lambda_{1..q} <- T(eta)^T lambda_{1..q};
//   INIT      D_1 = h0 f(y) folds into lambda_0, higher rows reset.
// M = I - c_M J(y_J) is a constant of the map (the recorded y_J and the
// forward's rate constants); the backward re-forms and re-factors it from the
// REFACTOR row each time the walk enters another REFACTOR's range.

// lambda_{1..q} <- T(eta)^T lambda_{1..q}: lambda'_m = sum_{i<=m} T_im lambda_i
template <int KS>
__device__ __forceinline__ void rescale_adjoint(double (&L)[NROW][KS], int q, double eta, const double *coef, int lane) {
  double tv = 0.0;
  if (lane < QMAX * QMAX) {
    const double *cp = coef + lane * (QMAX + 1);
    tv = __ldg(cp + QMAX);
#pragma unroll
    for (int p = QMAX - 1; p >= 0; --p) tv = fma(tv, eta, __ldg(cp + p));
  }
  // m descending: row m reads rows i <= m, still unchanged
#pragma unroll
  for (int mm = QMAX; mm >= 1; --mm) {
    if (mm > q) continue;
    double nl[KS];
#pragma unroll
    for (int k = 0; k < KS; ++k) nl[k] = 0.0;
#pragma unroll
    for (int i = 1; i <= QMAX; ++i) {
      if (i > mm) continue;
      const double t = __shfl_sync(FULL, tv, (i - 1) * QMAX + (mm - 1));
#pragma unroll
      for (int k = 0; k < KS; ++k) nl[k] = fma(t, L[i][k], nl[k]);
    }
#pragma unroll
    for (int k = 0; k < KS; ++k) L[mm][k] = nl[k];
  }
}

// Adjoint of an accepted STEP at order q (before the implicit part):
// lambda_d = lambda_{q+2} + lambda_{q+1} + sum_{m<=q} lambda_m; lambda_i (i<=q)
// = prefix sums, lambda_{q+1} = -lambda_{q+2}, lambda_{q+2} = 0.
template <int KS>
__device__ __forceinline__ void step_adjoint_linear(double (&L)[NROW][KS], int q, double (&lamd)[KS]) {
#define CHEM_ADJ_CASE(Q_)                                                           \
  case Q_:                                                                         \
    _Pragma("unroll") for (int k = 0; k < KS; ++k) {                               \
      double acc = 0.0;                                                            \
      _Pragma("unroll") for (int m = 0; m <= Q_; ++m) {                            \
        acc += L[m][k];                                                            \
        L[m][k] = acc;                                                             \
      }                                                                            \
      lamd[k] = L[Q_ + 2][k] + L[Q_ + 1][k] + acc;                                 \
      L[Q_ + 1][k] = -L[Q_ + 2][k];                                                \
      L[Q_ + 2][k] = 0.0;                                                          \
    }                                                                              \
    break;
  switch (q) {
    CHEM_ADJ_CASE(1) CHEM_ADJ_CASE(2) CHEM_ADJ_CASE(3) CHEM_ADJ_CASE(4) CHEM_ADJ_CASE(5)
    default:
      break;
  }
#undef CHEM_ADJ_CASE
}

// rates RT and partials PP = dr_j/dy_l at the y stored in Wd[Y]
template <int KS>
__device__ __forceinline__ void rates_partials(const MechDev &M, const Tabs &tb, double *Wd, int lane) {
  unsigned char *wd = reinterpret_cast<unsigned char *>(Wd);
  for (int j = lane; j < M.R; j += WARP) {
    const uint2 sl = tab<uint2>(tb, M.tab.rx_slots)[j];
    double r = Wd[M.d_KT + j] * at<double>(wd, sl.x & 0xffff);
    if (M.max_reac > 1) r *= at<double>(wd, sl.x >> 16);
    if (M.max_reac > 2) r *= at<double>(wd, sl.y & 0xffff);
    Wd[M.d_RT + j] = r;
  }
  for (int pr = lane; pr < M.n_pairs; pr += WARP) {
    const int j = tab<int>(tb, M.tab.pair_rx)[pr];
    const unsigned o = tab<unsigned>(tb, M.tab.pair_other)[pr];
    double p = Wd[M.d_KT + j];
    if (M.max_reac > 1) p *= at<double>(wd, o & 0xffff);
    if (M.max_reac > 2) p *= at<double>(wd, o >> 16);
    Wd[M.a_PP + pr] = p;
  }
  __syncwarp();
}

// Wd[MU] = v; runs nu.mu and J^T mu programs; theta gradient += scale * r_j * (nu_j . v); out = J^T v
template <int KS>
__device__ __forceinline__ void jt_and_theta(const MechDev &M, double *Wd, const bool (&own)[KS], const double (&v)[KS],
                                             double scale, double (&out)[KS], int lane) {
#pragma unroll
  for (int k = 0; k < KS; ++k)
    if (own[k]) Wd[M.a_MU + lane + WARP * k] = v[k];
  __syncwarp();
  run_prog<double, false, false, true, false>(M.nudot_ops, M.nudot_runs, M.nudot_nruns, M.nudot_npass, Wd, lane);
  run_prog<double, false, false, true, false>(M.jt_ops, M.jt_runs, M.jt_nruns, M.jt_npass, Wd, lane);
  for (int j = lane; j < M.R; j += WARP) Wd[M.a_G + j] = fma(scale * Wd[M.d_RT + j], Wd[M.a_NM + j], Wd[M.a_G + j]);
#pragma unroll
  for (int k = 0; k < KS; ++k) out[k] = own[k] ? Wd[M.a_JTM + lane + WARP * k] : 0.0;
  __syncwarp();
}

template <int KS>
__device__ __forceinline__ void read_row(const double *yt, int r, int S, const bool (&own)[KS], int lane, double (&y)[KS]) {
#pragma unroll
  for (int k = 0; k < KS; ++k) y[k] = own[k] ? yt[(int64_t)r * S + lane + WARP * k] : 0.0;
}

template <int KS>
__device__ void backward_cell(const MechDev &M, const CellsDev &C, const AdjDev &A, const SolveParams &P, const Tabs &tb,
                              double *Wd, double *WL, const int lane, const int64_t cell) {
  const int64_t NC = C.n_cells;
  Cell<double, KS, false> cl(M, P, tb, Wd, WL, lane);
  cl.init_constants();
  unsigned char *wd = reinterpret_cast<unsigned char *>(Wd);
  for (int k = lane; k < M.a_nconst; k += WARP) at<double>(wd, __ldg(M.a_const_off + k)) = __ldg(M.a_const_val + k);
  for (int j = lane; j < M.R; j += WARP) Wd[M.a_G + j] = 0.0;
  double y0[KS];
  load_cell<KS>(M, C, Wd, lane, cell, cl.own, y0);   // rate constants
  double L[NROW][KS];
#pragma unroll
  for (int m = 0; m < NROW; ++m)
#pragma unroll
    for (int k = 0; k < KS; ++k) L[m][k] = 0.0;
#pragma unroll
  for (int k = 0; k < KS; ++k) L[0][k] = cl.own[k] ? A.dLdy[(int64_t)(lane + WARP * k) * NC + cell] : 0.0;

  const int n = C.tape_n[cell];
  const int *kqs = C.tape_kq + cell * (int64_t)C.tape_cap;
  const double *vals = C.tape_val + cell * (int64_t)C.tape_cap;
  const double *yt = C.ytape + cell * (int64_t)C.row_cap * M.S;
  int row = C.tape_rows[cell];     // rows of the events before the walk position
  // the walk reads rows row-1, row-2, ...; the next one is loaded a row ahead
  // (its global loads complete while the current event is processed)
  double pre[KS];
  int pre_row = row - 1;
  if (pre_row >= 0) read_row<KS>(yt, pre_row, M.S, cl.own, lane, pre);
  auto take_row = [&](double (&y)[KS]) {      // row (already decremented)
    if (pre_row == row) {
#pragma unroll
      for (int k = 0; k < KS; ++k) y[k] = pre[k];
    } else {
      read_row<KS>(yt, row, M.S, cl.own, lane, y);
    }
    pre_row = row - 1;
    if (pre_row >= 0) read_row<KS>(yt, pre_row, M.S, cl.own, lane, pre);
  };
  int er = n - 1;                  // the last REFACTOR before the walk position
  while (er >= 0 && (__ldg(kqs + er) & 0xff) != EV_REFACTOR) --er;
  int m_event = -1;                // the REFACTOR whose LU is in WL
  double lamd[KS], lyp[KS], lpsi[KS];
#pragma unroll
  for (int k = 0; k < KS; ++k) lamd[k] = lyp[k] = lpsi[k] = 0.0;
  int sq = 1;
  double sc = 0.0, ss = 1.0;
  bool bad = false;

  for (int e = n - 1; e >= 0; --e) {
    const int kq = __ldg(kqs + e);
    const double val = __ldg(vals + e);
    const int kind = kq & 0xff, q = kq >> 8;
    if (kind == EV_RESCALE) {
      rescale_adjoint<KS>(L, q, val, M.rescale_coef, lane);
    } else if (kind == EV_STEP) {
      step_adjoint_linear<KS>(L, q, lamd);
#pragma unroll
      for (int k = 0; k < KS; ++k) lyp[k] = lpsi[k] = 0.0;
      sq = q;
      sc = val;
      while (er >= e) {
        --er;
        while (er >= 0 && (__ldg(kqs + er) & 0xff) != EV_REFACTOR) --er;
      }
      if (er < 0) {
        bad = true;
        break;
      }
      const double cM = __ldg(vals + er);
      if (er != m_event) {
        double yJ[KS];
        read_row<KS>(yt, __ldg(kqs + er) >> 8, M.S, cl.own, lane, yJ);
        cl.form_and_factor(cM, yJ);
        m_event = er;
      }
      ss = (sc == cM) ? 1.0 : 2.0 * recip_nr(fma(sc, recip_nr(cM), 1.0));   // as the forward formed it
    } else if (kind == EV_PROJECT) {
#pragma unroll
      for (int k = 0; k < KS; ++k)
        if (q == lane + WARP * k) {
          lyp[k] = -lamd[k];
          lamd[k] = 0.0;
        }
    } else if (kind == EV_ITER) {
      if (--row < 0) {
        bad = true;
        break;
      }
      double y[KS], g[KS], jtg[KS];
      take_row(y);
#pragma unroll
      for (int k = 0; k < KS; ++k)
        if (cl.own[k]) Wd[M.d_Y + lane + WARP * k] = y[k];
      __syncwarp();
      rates_partials<KS>(M, tb, Wd, lane);
      // g = s M^{-T} lambda_d
#pragma unroll
      for (int k = 0; k < KS; ++k)
        if (cl.own[k]) Wd[M.d_Y + cl.pos[k]] = lamd[k];   // the solve vector: y's slots (y was consumed)
      __syncwarp();
      run_prog<double, false, false, false, false>(M.fwdT_ops, M.fwdT_runs, M.fwdT_nruns, M.fwdT_npass, Wd, lane);
      run_prog<double, false, false, false, false>(M.bwdT_ops, M.bwdT_runs, M.bwdT_nruns, M.bwdT_npass, Wd, lane);
#pragma unroll
      for (int k = 0; k < KS; ++k) g[k] = cl.own[k] ? -ss * Wd[M.d_Y + cl.pos[k]] : 0.0;   // the programs leave -M^{-T} lambda
      __syncwarp();
      jt_and_theta<KS>(M, Wd, cl.own, g, sc, jtg, lane);
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        const double cj = sc * jtg[k];
        lamd[k] += cj - g[k];
        lyp[k] += cj;
        lpsi[k] -= g[k];
      }
      if (q == 0) {
        // the predictor: y_pred = sum_{m<=q} D_m, psi = (1/gamma_q) sum gamma_m D_m
        const double iq = c_igam[sq];
#pragma unroll
        for (int m = 0; m <= QMAX; ++m) {
          if (m > sq) continue;
          const double gm = (m >= 1) ? c_gam[m] * iq : 0.0;
#pragma unroll
          for (int k = 0; k < KS; ++k) L[m][k] += fma(gm, lpsi[k], lyp[k]);
        }
      }
    } else if (kind == EV_REFACTOR) {
      --row;
    } else if (kind == EV_INIT) {
      // D_0 = y, D_1 = h0 f(y), higher rows reset
      if (--row < 0) {
        bad = true;
        break;
      }
      double y[KS], jtl[KS], l1[KS];
      take_row(y);
#pragma unroll
      for (int k = 0; k < KS; ++k)
        if (cl.own[k]) Wd[M.d_Y + lane + WARP * k] = y[k];
      __syncwarp();
      rates_partials<KS>(M, tb, Wd, lane);
#pragma unroll
      for (int k = 0; k < KS; ++k) l1[k] = L[1][k];
      jt_and_theta<KS>(M, Wd, cl.own, l1, val, jtl, lane);
#pragma unroll
      for (int k = 0; k < KS; ++k) L[0][k] = fma(val, jtl[k], L[0][k]);
#pragma unroll
      for (int m = 1; m < NROW; ++m)
#pragma unroll
        for (int k = 0; k < KS; ++k) L[m][k] = 0.0;
    }
  }
#pragma unroll
  for (int k = 0; k < KS; ++k)
    if (cl.own[k]) A.dLdy0[(int64_t)(lane + WARP * k) * NC + cell] = bad ? 0.0 : L[0][k];
  for (int j = lane; j < M.R; j += WARP) A.gcell[(int64_t)j * NC + cell] = bad ? 0.0 : Wd[M.a_G + j];
  if (bad && lane == 0) C.tape_bad[cell] = 1;
}

template <int KS>
__global__ void __launch_bounds__(MAX_WARPS_PER_BLOCK * WARP) adjoint_kernel(const __grid_constant__ MechDev M, const CellsDev C, const AdjDev A,
                                                                    const SolveParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & (WARP - 1);
  const int warp = threadIdx.x / WARP;
  Tabs tb;
  tb.base = tb.gbase = M.blob[0];
  double *Wd = reinterpret_cast<double *>(smem + (size_t)warp * P.cell_bytes);
  double *WL = Wd + P.wd_pad;
  // with a queue, every warp takes the next slot of C.order (longest tapes
  // first) until none is left; without one, slot = its global warp index
  for (int64_t slot = (int64_t)blockIdx.x * P.warps_per_block + warp;;) {
    if (C.queue) {
      long long q = 0;
      if (lane == 0) q = (long long)atomicAdd(C.queue, 1ull);
      slot = __shfl_sync(FULL, q, 0);
    }
    if (slot >= C.n_cells) break;
    const int64_t cell = C.order ? (int64_t)C.order[slot] : slot;
    if (C.tape_bad[cell]) {
      for (int i = lane; i < M.S; i += WARP) A.dLdy0[(int64_t)i * C.n_cells + cell] = 0.0;
      for (int j = lane; j < M.R; j += WARP) A.gcell[(int64_t)j * C.n_cells + cell] = 0.0;
    } else {
      backward_cell<KS>(M, C, A, P, tb, Wd, WL, lane, cell);
    }
    __syncwarp();
    if (!C.queue) break;
  }
}

// ---------------------------------------------------------------- tangent
// Forward-mode derivative of the same frozen-control map the adjoint
// differentiates: one warp per cell walks its tape forward carrying the
// tangent dD of the history in registers.  The iterations need
// c (J(y_k) v + F_theta(y_k) dtheta) - dpsi - dd, and J v + F_theta dtheta is
// the f program applied to s_j = k~_j sum_s (prod_{s' != s} y) v_s + r_j dtheta_j
// in place of the rates r_j; then one solve with the REFACTOR's LU.

// f-program image of J(y) v + F_theta dtheta; y in Wd[Y], v in Wd[a_MU]
template <int KS>
__device__ __forceinline__ void tangent_f(const MechDev &M, const Tabs &tb, double *Wd, const double *dtheta,
                                          const bool (&own)[KS], const double (&v)[KS], double (&out)[KS], int lane) {
#pragma unroll
  for (int k = 0; k < KS; ++k)
    if (own[k]) Wd[M.a_MU + lane + WARP * k] = v[k];
  __syncwarp();
  unsigned char *wd = reinterpret_cast<unsigned char *>(Wd);
  const unsigned dv = (unsigned)(M.a_MU - M.d_Y) * 8u;      // from y_l to v_l
  for (int j = lane; j < M.R; j += WARP) {
    const uint2 sl = tab<uint2>(tb, M.tab.rx_slots)[j];
    const unsigned o1 = sl.x & 0xffff, o2 = sl.x >> 16, o3 = sl.y & 0xffff;
    const int nr = __ldg(M.rx_nreac + j);
    const double kt = Wd[M.d_KT + j];
    const double y1 = at<double>(wd, o1), v1 = at<double>(wd, o1 + dv);
    double sv, r;
    if (nr == 1) {
      sv = v1;
      r = y1;
    } else {
      const double y2 = at<double>(wd, o2), v2 = at<double>(wd, o2 + dv);
      if (nr == 2) {
        sv = v1 * y2 + y1 * v2;
        r = y1 * y2;
      } else {
        const double y3 = at<double>(wd, o3), v3 = at<double>(wd, o3 + dv);
        sv = v1 * y2 * y3 + y1 * v2 * y3 + y1 * y2 * v3;
        r = y1 * y2 * y3;
      }
    }
    double sj = kt * sv;
    if (dtheta) sj = fma(kt * r, dtheta[j], sj);
    Wd[M.d_RT + j] = sj;
  }
  __syncwarp();
  run_prog<double, false, false, true, false>(tab<ushort4>(tb, M.tab.f_ops), tab<uint32_t>(tb, M.tab.f_runs), M.f_nruns,
                                              M.f_npass, Wd, lane);
#pragma unroll
  for (int k = 0; k < KS; ++k) out[k] = own[k] ? Wd[M.d_F + lane + WARP * k] : 0.0;
  __syncwarp();
}

template <int KS>
__device__ void tangent_cell(const MechDev &M, const CellsDev &C, const TanDev &A, const SolveParams &P, const Tabs &tb,
                             double *Wd, double *WL, const int lane, const int64_t cell) {
  const int64_t NC = C.n_cells;
  Cell<double, KS, false> cl(M, P, tb, Wd, WL, lane);
  cl.init_constants();
  double y0[KS];
  load_cell<KS>(M, C, Wd, lane, cell, cl.own, y0);   // rate constants
  double dD[NROW][KS];
#pragma unroll
  for (int m = 0; m < NROW; ++m)
#pragma unroll
    for (int k = 0; k < KS; ++k) dD[m][k] = 0.0;
#pragma unroll
  for (int k = 0; k < KS; ++k) dD[0][k] = cl.own[k] ? A.dy0[(int64_t)(lane + WARP * k) * NC + cell] : 0.0;
  const int n = C.tape_n[cell], nrows = C.tape_rows[cell];
  const int *kqs = C.tape_kq + cell * (int64_t)C.tape_cap;
  const double *vals = C.tape_val + cell * (int64_t)C.tape_cap;
  const double *yt = C.ytape + cell * (int64_t)C.row_cap * M.S;
  int row = 0;
  // the tape's rows are read in order; the next one is loaded a row ahead (its
  // global loads complete while the current event is processed)
  double pre[KS];
  if (nrows > 0) read_row<KS>(yt, 0, M.S, cl.own, lane, pre);
  auto next_row = [&](double (&y)[KS]) {
#pragma unroll
    for (int k = 0; k < KS; ++k) y[k] = pre[k];
    if (++row < nrows) read_row<KS>(yt, row, M.S, cl.own, lane, pre);
  };
  bool in_step = false, have_M = false, bad = false;
  double cM = 0.0, sc = 0.0, ss = 1.0;
  int sq = 1;
  double dyp[KS], dpsi[KS], dd[KS];
  bool pm[KS];
#pragma unroll
  for (int k = 0; k < KS; ++k) {
    dyp[k] = dpsi[k] = dd[k] = 0.0;
    pm[k] = false;
  }
  for (int e = 0; e < n; ++e) {
    const int kq = __ldg(kqs + e);
    const double val = __ldg(vals + e);
    const int kind = kq & 0xff, q = kq >> 8;
    if (!in_step && (kind == EV_ITER || kind == EV_PROJECT || kind == EV_STEP)) {
      // a step's events are its iterations, its projections, then the STEP (q, c):
      // read ahead to the STEP and form the predictor's tangent
      int es = e;
      for (; es < n; ++es) {
        const int kq2 = __ldg(kqs + es);
        if ((kq2 & 0xff) == EV_STEP) break;
        if ((kq2 & 0xff) == EV_PROJECT) {
#pragma unroll
          for (int k = 0; k < KS; ++k)
            if ((kq2 >> 8) == lane + WARP * k) pm[k] = true;
        }
      }
      if (es >= n || !have_M) {
        bad = true;
        break;
      }
      sq = __ldg(kqs + es) >> 8;
      sc = __ldg(vals + es);
      ss = (sc == cM) ? 1.0 : 2.0 * recip_nr(fma(sc, recip_nr(cM), 1.0));   // as the forward formed it
      const double iq = c_igam[sq];
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        dyp[k] = dD[0][k];
        dpsi[k] = 0.0;
        dd[k] = 0.0;
      }
#pragma unroll
      for (int m = 1; m <= QMAX; ++m) {
        if (m > sq) continue;
        const double gm = c_gam[m];
#pragma unroll
        for (int k = 0; k < KS; ++k) {
          dyp[k] += dD[m][k];
          dpsi[k] = fma(gm, dD[m][k], dpsi[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < KS; ++k) dpsi[k] *= iq;
      in_step = true;
    }
    if (kind == EV_RESCALE) {
      rescale<KS>(dD, q, val, M.rescale_coef, lane);
    } else if (kind == EV_INIT) {
      // D_0 = y, D_1 = h0 f(y), higher rows reset
      if (row >= nrows) {
        bad = true;
        break;
      }
      double y[KS], g[KS], d0[KS];
      next_row(y);
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        d0[k] = dD[0][k];
        if (cl.own[k]) Wd[M.d_Y + lane + WARP * k] = y[k];
      }
      tangent_f<KS>(M, tb, Wd, A.dtheta, cl.own, d0, g, lane);
#pragma unroll
      for (int m = 1; m < NROW; ++m)
#pragma unroll
        for (int k = 0; k < KS; ++k) dD[m][k] = 0.0;
#pragma unroll
      for (int k = 0; k < KS; ++k) dD[1][k] = val * g[k];
    } else if (kind == EV_REFACTOR) {
      // the iteration matrix of the recorded run (a constant of the map)
      if (row >= nrows) {
        bad = true;
        break;
      }
      double yJ[KS];
      next_row(yJ);
      cl.form_and_factor(val, yJ);
      cM = val;
      have_M = true;
    } else if (kind == EV_ITER) {
      if (row >= nrows) {
        bad = true;
        break;
      }
      double y[KS], v[KS], g[KS], b[KS], x[KS];
      next_row(y);
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        v[k] = dyp[k] + dd[k];
        if (cl.own[k]) Wd[M.d_Y + lane + WARP * k] = y[k];
      }
      tangent_f<KS>(M, tb, Wd, A.dtheta, cl.own, v, g, lane);
#pragma unroll
      for (int k = 0; k < KS; ++k) b[k] = sc * g[k] - dpsi[k] - dd[k];
      cl.solve(b, x);
#pragma unroll
      for (int k = 0; k < KS; ++k) dd[k] = fma(ss, x[k], dd[k]);
    } else if (kind == EV_STEP) {
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        if (pm[k]) dd[k] = -dyp[k];          // projected onto y = 0
        pm[k] = false;
      }
      accept_update<KS>(dD, sq, dd);
      in_step = false;
    }
    // PROJECT events were read with their step's predictor
  }
#pragma unroll
  for (int k = 0; k < KS; ++k)
    if (cl.own[k]) A.dy[(int64_t)(lane + WARP * k) * NC + cell] = bad ? 0.0 : dD[0][k];
  if (bad && lane == 0) C.tape_bad[cell] = 1;
}

template <int KS>
__global__ void __launch_bounds__(TAN_WARPS_PER_BLOCK * WARP) tangent_kernel(const __grid_constant__ MechDev M, const CellsDev C,
                                                                    const TanDev A, const SolveParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & (WARP - 1);
  const int warp = threadIdx.x / WARP;
  Tabs tb;
  tb.base = tb.gbase = M.blob[0];
  double *Wd = reinterpret_cast<double *>(smem + (size_t)warp * P.cell_bytes);
  double *WL = Wd + P.wd_pad;
  for (int64_t slot = (int64_t)blockIdx.x * P.warps_per_block + warp;;) {   // as in adjoint_kernel
    if (C.queue) {
      long long q = 0;
      if (lane == 0) q = (long long)atomicAdd(C.queue, 1ull);
      slot = __shfl_sync(FULL, q, 0);
    }
    if (slot >= C.n_cells) break;
    const int64_t cell = C.order ? (int64_t)C.order[slot] : slot;
    if (C.tape_bad[cell]) {
      for (int i = lane; i < M.S; i += WARP) A.dy[(int64_t)i * C.n_cells + cell] = 0.0;
    } else {
      tangent_cell<KS>(M, C, A, P, tb, Wd, WL, lane, cell);
    }
    __syncwarp();
    if (!C.queue) break;
  }
}

// Dynamic shared memory of a block of `smem` bytes, padded so that no more
// than bps such blocks fit on one SM (blocks per SM by shared memory:
// floor(per-SM capacity / (block's bytes + the per-block reservation))).
size_t pad_smem_to_blocks(size_t smem, int bps) {
  int dev = 0, per_sm = 0, reserved = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (bps < 1 || per_sm <= 0) return smem;
  const long need = (long)per_sm / (long)(bps + 1) - (long)reserved + 1;    // bps + 1 blocks no longer fit
  size_t s = need > (long)smem ? (size_t)need : smem;
  s = (s + 127) & ~(size_t)127;
  return s <= (size_t)optin ? s : smem;
}

// Launch shape of a walk kernel.  A walk's cells each take one warp (the queue
// hands out the longest tapes first), so while the batch has fewer than
// NARROW_CELLS_PER_WARP cells per warp at NARROW_WARPS_PER_SM warps per SM,
// nearly every cell has a warp of its own and the walk lasts as long as its
// slowest cells, which run faster with fewer warps beside them on the SM: such
// batches run at most NARROW_WARPS_PER_SM warps per SM (2,048 cells of the
// 72-species mechanism: tangent 12.3 -> 11.2 ms, adjoint 12.5 -> 11.3 ms);
// larger ones at the occupancy that keeps the most cells resident (shared
// memory bounds it), ties to the larger block (fewer blocks to place).  Blocks
// per SM are bounded by padding each block's shared memory, so the block
// scheduler cannot stack a third block of a two-block shape on one SM while
// another SM has none.  The kernel's dynamic shared-memory limit must be
// raised first.
constexpr int NARROW_WARPS_PER_SM = 8;
constexpr int NARROW_CELLS_PER_WARP = 2;

bool narrow_batch(int64_t n_cells) {
  int dev = 0, n_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  return n_cells < (int64_t)NARROW_CELLS_PER_WARP * NARROW_WARPS_PER_SM * n_sm;
}

struct WalkShape {
  int warps_per_block = 0;
  int blocks_per_sm = 0;
  size_t smem = 0;        // dynamic shared memory per block (>= warps_per_block * cell_bytes)
};

template <typename K>
WalkShape walk_shape(K kernel, int cell_bytes, int max_warps, int64_t n_cells) {
  WalkShape ws;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const bool narrow = narrow_batch(n_cells);
  int best_w = 0, best_cells = 0, best_nb = 0;
  for (int w = 1; w <= max_warps && (long)w * cell_bytes <= (long)optin; ++w) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, w * WARP, (size_t)w * cell_bytes) != cudaSuccess)
      continue;
    int cells = w * nb;
    if (narrow && cells > NARROW_WARPS_PER_SM) {
      // the most whole blocks of w warps within the narrow bound
      nb = NARROW_WARPS_PER_SM / w;
      cells = w * nb;
    }
    if (cells >= best_cells && cells > 0) {
      best_cells = cells;
      best_w = w;
      best_nb = nb;
    }
  }
  if (best_w < 1) return ws;
  ws.warps_per_block = best_w;
  ws.blocks_per_sm = best_nb;
  ws.smem = (size_t)best_w * cell_bytes;
  int natural = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&natural, kernel, best_w * WARP, ws.smem) == cudaSuccess &&
      natural > best_nb)
    ws.smem = pad_smem_to_blocks(ws.smem, best_nb);
  return ws;
}

// Grid of a walk launch: with the queue, the resident blocks of the shape on
// every SM (never more than the cells need); without, one warp per cell.
int walk_blocks(const CellsDev &C, int warps_per_block, int blocks_per_sm) {
  const int64_t need = (C.n_cells + warps_per_block - 1) / warps_per_block;
  if (!C.queue) return (int)need;
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t full = (int64_t)n_sm * (blocks_per_sm > 0 ? blocks_per_sm : 1);
  return (int)(full < need ? full : need);
}

template <int KS>
cudaError_t launch_tan_t(const MechDev &M, const CellsDev &C, const TanDev &A, const SolveParams &P0, cudaStream_t stream) {
  cudaError_t e = allow_max_smem<tangent_kernel<KS>>();
  if (e != cudaSuccess) return e;
  SolveParams P = P0;
  const WalkShape ws = walk_shape(tangent_kernel<KS>, P.cell_bytes, TAN_WARPS_PER_BLOCK, C.n_cells);
  if (ws.warps_per_block < 1) return cudaErrorInvalidValue;
  P.warps_per_block = ws.warps_per_block;
  const int blocks = walk_blocks(C, P.warps_per_block, ws.blocks_per_sm);
  tangent_kernel<KS><<<blocks, P.warps_per_block * WARP, ws.smem, stream>>>(M, C, A, P);
  return cudaGetLastError();
}

// dL/dtheta_j = sum over cells of the per-cell gradients, in cell order (added
// to out[j] when accumulating over the steps of a checkpointed backward)
__global__ void theta_reduce_kernel(const double *gcell, int64_t n_cells, int R, double *out, int accumulate) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= R) return;
  double s = 0.0;
  for (int64_t c = 0; c < n_cells; ++c) s += gcell[(int64_t)j * n_cells + c];
  out[j] = accumulate ? out[j] + s : s;
}

__global__ void count_flags_kernel(const int *flag, int64_t n, unsigned long long *acc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned v = __reduce_add_sync(FULL, (i < n && flag[i] != 0) ? 1u : 0u);
  if ((threadIdx.x & (WARP - 1)) == 0 && v) atomicAdd(acc, (unsigned long long)v);
}

template <int KS>
cudaError_t launch_adj_t(const MechDev &M, const CellsDev &C, const AdjDev &A, const SolveParams &P0, cudaStream_t stream) {
  cudaError_t e = allow_max_smem<adjoint_kernel<KS>>();
  if (e != cudaSuccess) return e;
  SolveParams P = P0;
  const WalkShape ws = walk_shape(adjoint_kernel<KS>, P.cell_bytes, ADJ_WARPS_PER_BLOCK, C.n_cells);
  if (ws.warps_per_block < 1) return cudaErrorInvalidValue;
  P.warps_per_block = ws.warps_per_block;
  const int blocks = walk_blocks(C, P.warps_per_block, ws.blocks_per_sm);
  adjoint_kernel<KS><<<blocks, P.warps_per_block * WARP, ws.smem, stream>>>(M, C, A, P);
  return cudaGetLastError();
}

// ----------------------------------------------------------- queue order
// One warp per cell computes a cost key; the queue then hands out the most
// expensive cells first, so that the slowest solves do not start last (with a
// few cells per warp, one late expensive cell otherwise holds a whole SM).
// The key is the cell's cost in the previous solve of the batch (the f
// evaluations, solves, factorisations and steps of its statistics, weighted
// by their FP64 work), and for a batch's first solve the sum of the cell's
// rate constants k~_j: air density (every bimolecular rate scales with it),
// temperature and light set how fast and stiff the cell's chemistry is, while
// its concentrations (drawn at random in a fresh state) say little about the
// work ahead.  Measured on the 10,000-cell workload's first solve: ordered by
// this key 30 ms, by the stiffness ratio ||f(y0)|| / ||y0|| 35 ms, by the
// exact costs 28 ms.  The keys (log2) are then bucketed linearly between the
// batch's smallest and largest key into ORDER_BUCKETS - 1 buckets, most
// expensive first, and counting-sorted.

// float -> unsigned int, monotone: the larger float gives the larger integer
__device__ __forceinline__ unsigned ordered_bits(float f) {
  const unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_ordered_bits(unsigned u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// keys: bucket[cell] receives the key's bits (float); hist[2 ORDER_BUCKETS]
// the largest key's ordered bits, hist[2 ORDER_BUCKETS + 1] the complement of
// the smallest's (both start at 0); a cell with bad inputs gets -inf
template <int KS>
__global__ void __launch_bounds__(ORDER_WARPS * WARP) order_keys_kernel(const __grid_constant__ MechDev M, const CellsDev C,
                                                                          const SolveParams P, int *bucket, int *hist) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & (WARP - 1);
  const int warp = threadIdx.x / WARP;
  const int64_t cell = (int64_t)blockIdx.x * ORDER_WARPS + warp;
  if (cell >= C.n_cells) return;
  double *Wd = reinterpret_cast<double *>(smem + (size_t)warp * P.cell_bytes);
  float l = -INFINITY;                        // log2 of the key, larger first
  const chem_cell_stats prev = C.stats[cell];
  if (prev.steps > 0) {
    l = (float)log2(65.0 * prev.f_evals + 100.0 * prev.solves + 560.0 * prev.jac_evals + 150.0 * prev.steps);
  } else {
    bool own[KS];
#pragma unroll
    for (int k = 0; k < KS; ++k) own[k] = lane + WARP * k < M.S;
    double y0[KS];
    if (!load_cell<KS>(M, C, Wd, lane, cell, own, y0)) {
      double sk = 0.0;
      for (int j = lane; j < M.R; j += WARP) sk += Wd[M.d_KT + j];
      sk = warp_sum(sk);
      if (sk > 0.0 && isfinite(sk)) l = (float)log2(sk);
    }
  }
  if (lane == 0) {
    bucket[cell] = __float_as_int(l);
    if (isfinite(l)) {
      atomicMax(reinterpret_cast<unsigned *>(hist) + 2 * ORDER_BUCKETS, ordered_bits(l));
      atomicMax(reinterpret_cast<unsigned *>(hist) + 2 * ORDER_BUCKETS + 1, ~ordered_bits(l));
    }
  }
}

// the keys into buckets 0 .. ORDER_BUCKETS - 2, largest key first, linearly
// over the batch's range; bad inputs last
__global__ void order_bucket_kernel(int *bucket, int *hist, int64_t n) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const float l = __int_as_float(bucket[c]);
  int b = ORDER_BUCKETS - 1;
  if (isfinite(l)) {
    const float hi = from_ordered_bits(reinterpret_cast<const unsigned *>(hist)[2 * ORDER_BUCKETS]);
    const float lo = from_ordered_bits(~reinterpret_cast<const unsigned *>(hist)[2 * ORDER_BUCKETS + 1]);
    b = hi > lo ? (int)((hi - l) / (hi - lo) * (float)(ORDER_BUCKETS - 2)) : 0;
    b = b < 0 ? 0 : (b > ORDER_BUCKETS - 2 ? ORDER_BUCKETS - 2 : b);
  }
  bucket[c] = b;
  atomicAdd(hist + b, 1);
}

// For the adjoint and tangent walks: the cells by the length of their tapes,
// longest first (the walk's work is proportional to it), so that the blocks the
// hardware dispatches last hold the shortest walks.
__global__ void order_tape_keys_kernel(const CellsDev C, int *bucket, int *hist) {
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= C.n_cells) return;
  const int n = C.tape_n[cell];
  int b = ORDER_BUCKETS - 1;
  if (n > 0) {
    const int k = (int)fmin(floor(8.0 * log2((double)n)), 254.0);   // 8 buckets per octave
    b = 254 - k;
  }
  bucket[cell] = b;
  atomicAdd(hist + b, 1);
}

// Coupled groups of G consecutive cells (which share their statistics): the
// groups by their cost in the previous solve, largest first; groups without
// one first, in group order.
__global__ void order_group_keys_kernel(const CellsDev C, int G, int64_t n_groups, int *bucket, int *hist) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_groups) return;
  const chem_cell_stats prev = C.stats[g * G];
  int b = 0;
  if (prev.steps > 0) {
    const double l = log2(65.0 * prev.f_evals + 100.0 * prev.solves + 560.0 * prev.jac_evals + 150.0 * prev.steps);
    const int k = (int)fmin(fmax(floor(4.0 * l), -126.0), 126.0);
    b = 128 - k;
  }
  bucket[g] = b;
  atomicAdd(hist + b, 1);
}

// exclusive prefix sum of the bucket counts into the scatter cursors
__global__ void order_scan_kernel(int *hist) {
  if (threadIdx.x != 0) return;
  int acc = 0;
  for (int b = 0; b < ORDER_BUCKETS; ++b) {
    const int n = hist[b];
    hist[ORDER_BUCKETS + b] = acc;
    acc += n;
  }
}

__global__ void order_scatter_kernel(const int *bucket, int *hist, int *order, int64_t n) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int pos = atomicAdd(hist + ORDER_BUCKETS + bucket[c], 1);
  order[pos] = (int)c;
}

template <int KS>
cudaError_t launch_order_t(const MechDev &M, const CellsDev &C, const SolveParams &P, int *bucket, int *hist, cudaStream_t s) {
  const size_t smem = (size_t)P.cell_bytes * ORDER_WARPS;
  cudaError_t e = allow_max_smem<order_keys_kernel<KS>>();
  if (e != cudaSuccess) return e;
  const int64_t blocks = (C.n_cells + ORDER_WARPS - 1) / ORDER_WARPS;
  order_keys_kernel<KS><<<(unsigned)blocks, ORDER_WARPS * WARP, smem, s>>>(M, C, P, bucket, hist);
  return cudaGetLastError();
}

// ----------------------------------------------------- derivative only
// a2 for every cell with the rate constants given (kt[R][C]): a block of
// GATHER_CELLS cells copies the hot table prefix into shared memory, reads its
// y and k~ tiles with the cells fastest (coalesced), transposes them into the
// cells' Wd slices, runs the rates and the f program one warp per cell, and
// writes f back the same way.
constexpr int GATHER_CELLS = 16;

template <int KS>
__global__ void __launch_bounds__(GATHER_CELLS * WARP) deriv_gather_kernel(const __grid_constant__ MechDev M, const int64_t NC,
                                                                             const double *kt, const double *y, double *f,
                                                                             const int cell_doubles) {
  extern __shared__ __align__(16) unsigned char smem[];
  // the hot table prefix (f program, reactant slots), then the cells' slices
  const int tb = M.tab.staged;
  for (int i = threadIdx.x; i < tb / 16; i += blockDim.x)
    reinterpret_cast<uint4 *>(smem)[i] = __ldg(reinterpret_cast<const uint4 *>(M.blob[0]) + i);
  double *sm = reinterpret_cast<double *>(smem + tb);
  const int lane = threadIdx.x & (WARP - 1);
  const int warp = threadIdx.x / WARP;
  const int64_t c0 = (int64_t)blockIdx.x * GATHER_CELLS;
  const int nb = (int)((NC - c0) < GATHER_CELLS ? (NC - c0) : GATHER_CELLS);    // cells of this block
  // tiles in: element (row, cell) -> slice of cell, slot row
  for (int i = threadIdx.x; i < M.S * GATHER_CELLS; i += blockDim.x) {
    const int r = i / GATHER_CELLS, cl = i % GATHER_CELLS;
    if (cl < nb) sm[(size_t)cl * cell_doubles + M.d_Y + r] = y[(int64_t)r * NC + c0 + cl];
  }
  for (int i = threadIdx.x; i < M.R * GATHER_CELLS; i += blockDim.x) {
    const int r = i / GATHER_CELLS, cl = i % GATHER_CELLS;
    if (cl < nb) sm[(size_t)cl * cell_doubles + M.d_KT + r] = kt[(int64_t)r * NC + c0 + cl];
  }
  if (warp < nb) {
    double *Wd = sm + (size_t)warp * cell_doubles;
    unsigned char *wd = reinterpret_cast<unsigned char *>(Wd);
    const unsigned char *gb = M.blob[0];
    for (int k = lane; k < M.d_nconst; k += WARP)
      at<double>(wd, reinterpret_cast<const int *>(gb + M.tab.dconst_off)[k]) = reinterpret_cast<const double *>(gb + M.tab.dconst_val)[k];
  }
  __syncthreads();
  if (warp < nb) f_core<true>(M, smem, sm + (size_t)warp * cell_doubles, lane);
  __syncthreads();
  for (int i = threadIdx.x; i < M.S * GATHER_CELLS; i += blockDim.x) {
    const int r = i / GATHER_CELLS, cl = i % GATHER_CELLS;
    if (cl < nb) f[(int64_t)r * NC + c0 + cl] = sm[(size_t)cl * cell_doubles + M.d_F + r];
  }
}

bool staged_driver(int driver) { return driver == CHEM_DRIVER_PERSISTENT; }

// Diagnostic: the solve kernels' warp sum of non-negative doubles, one warp
// per group of 32 consecutive elements of x.
__global__ void wsum_probe_kernel(const double *x, double *out, int64_t n_groups) {
  const int64_t g = (int64_t)blockIdx.x * (blockDim.x / WARP) + threadIdx.x / WARP;
  if (g >= n_groups) return;
  const int lane = threadIdx.x & (WARP - 1);
  const double s = warp_sum_nn(x[g * WARP + lane]);
  if (lane == 0) out[g] = s;
}

// Diagnostic: the solve kernels' FP64 reciprocal, element by element.
__global__ void recip_probe_kernel(const double *x, double *out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = recip_nr(x[i]);
}

}  // namespace

cudaError_t launch_wsum_probe(const double *x, double *out, int64_t n_groups, cudaStream_t stream) {
  if (n_groups <= 0) return cudaSuccess;
  wsum_probe_kernel<<<(unsigned)((n_groups + 7) / 8), 8 * WARP, 0, stream>>>(x, out, n_groups);
  return cudaGetLastError();
}

cudaError_t launch_recip_probe(const double *x, double *out, int64_t n, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  recip_probe_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(x, out, n);
  return cudaGetLastError();
}

size_t smem_per_cell(const MechDev &m, int lu_precision) {
  const size_t wd = (size_t)((m.Wd_len + 1) & ~1) * sizeof(double);
  const size_t wl = (size_t)m.WL_len * (lu_precision == 32 ? sizeof(float) : sizeof(double));
  return (wd + wl + 15) & ~(size_t)15;
}

size_t staged_bytes(const MechDev &m, int driver) { return staged_driver(driver) ? (size_t)m.tab.staged : 0; }

int max_warps_per_block(const MechDev &m, int lu_precision, int driver) {
  int dev = 0, smem_block = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const long avail = (long)smem_block - (long)staged_bytes(m, driver) - 64;
  const int w = avail > 0 ? (int)(avail / (long)smem_per_cell(m, lu_precision)) : 0;
  return w < MAX_WARPS_PER_BLOCK ? w : MAX_WARPS_PER_BLOCK;
}

cudaError_t set_constants() {
  double gam[QMAX + 2], igam[QMAX + 2];
  gam[0] = igam[0] = 0.0;
  for (int k = 1; k <= QMAX + 1; ++k) {
    double g = 0.0;
    for (int i = 1; i <= k; ++i) g += 1.0 / (double)i;
    gam[k] = g;
    igam[k] = 1.0 / g;
  }
  cudaError_t e = cudaMemcpyToSymbol(c_gam, gam, sizeof(gam));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_igam, igam, sizeof(igam));
}

int occupancy(const MechDev &M, int lu_precision, int driver, int warps_per_block) {
  const size_t smem = staged_bytes(M, driver) + smem_per_cell(M, lu_precision) * (size_t)warps_per_block;
  const bool f32 = lu_precision == 32;
  if (staged_driver(driver))
    return f32 ? occupancy_ks<float, true>(M, warps_per_block, smem) : occupancy_ks<double, true>(M, warps_per_block, smem);
  return f32 ? occupancy_ks<float, false>(M, warps_per_block, smem) : occupancy_ks<double, false>(M, warps_per_block, smem);
}

int best_warps_per_block(const MechDev &M, int lu_precision, int driver) {
  const int wmax = max_warps_per_block(M, lu_precision, driver);
  // The plain driver runs one cell per block: a block retires only when its
  // slowest cell does, and that tail costs more than the odd extra resident
  // cell a larger block may fit (72/186, 10,000 cells: 49.6 ms at 1 cell per
  // block against 64.1 ms at 11).
  if (!staged_driver(driver)) return (wmax >= 1 && occupancy(M, lu_precision, driver, 1) >= 1) ? 1 : 0;
  // The persistent driver stages the tables once per block: most resident
  // cells per SM, ties to the larger block.  (The walks' narrow-batch bound
  // was measured here too: a single first solve of 1,024 / 2,048 cells of the
  // 72/186 mechanism gains 10% / 8% at 8 cells per SM, but the four recorded
  // steps of the 2,048-cell differentiation workload lose 3%, 15.9 -> 16.4
  // ms: after the first step the queue is keyed by exact costs and the
  // throughput of the full occupancy wins.)
  int best_w = 0, best_cells = 0;
  for (int w = 1; w <= wmax; ++w) {
    const int cells = w * occupancy(M, lu_precision, driver, w);
    if (cells > 0 && cells >= best_cells) {
      best_cells = cells;
      best_w = w;
    }
  }
  return best_w;
}

cudaError_t launch_probe(const MechDev &M, const CellsDev &C, int lu_precision, int mode, double c, const double *y,
                         const double *b, double *out, cudaStream_t stream) {
  if (C.n_cells <= 0) return cudaSuccess;
  SolveParams P{};
  P.wd_pad = (M.Wd_len + 1) & ~1;
  P.cell_bytes = (int)smem_per_cell(M, lu_precision);
  P.warps_per_block = 1;
  P.prec = lu_precision == 32 ? 1 : 0;
  P.tab_bytes = 0;
  const bool f32 = lu_precision == 32;
  switch ((M.S + WARP - 1) / WARP) {
    case 1: return f32 ? launch_probe_t<float, 1>(M, C, P, mode, c, y, b, out, stream) : launch_probe_t<double, 1>(M, C, P, mode, c, y, b, out, stream);
    case 2: return f32 ? launch_probe_t<float, 2>(M, C, P, mode, c, y, b, out, stream) : launch_probe_t<double, 2>(M, C, P, mode, c, y, b, out, stream);
    case 3: return f32 ? launch_probe_t<float, 3>(M, C, P, mode, c, y, b, out, stream) : launch_probe_t<double, 3>(M, C, P, mode, c, y, b, out, stream);
    case 4: return f32 ? launch_probe_t<float, 4>(M, C, P, mode, c, y, b, out, stream) : launch_probe_t<double, 4>(M, C, P, mode, c, y, b, out, stream);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_solve(const MechDev &M, const CellsDev &C, const LaunchCfg &cfg, cudaStream_t stream) {
  if (C.n_cells <= 0) return cudaSuccess;
  SolveParams P;
  P.rtol = cfg.rtol;
  P.atol = cfg.atol;
  P.dt = cfg.dt;
  P.max_order = cfg.max_order;
  P.max_steps = cfg.max_steps;
  P.wd_pad = (M.Wd_len + 1) & ~1;
  P.cell_bytes = (int)smem_per_cell(M, cfg.lu_precision);
  P.warps_per_block = cfg.warps_per_block;
  P.prec = cfg.lu_precision == 32 ? 1 : 0;
  const bool staged = staged_driver(cfg.driver);
  P.tab_bytes = (int)staged_bytes(M, cfg.driver);
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  P.couple = cfg.couple > 1 ? cfg.couple : 1;
  P.stage_wait = cfg.stage_wait > 0 ? cfg.stage_wait : (cfg.stage_wait < 0 ? 0 : STAGE_WAIT_DEFAULT);
  if (P.warps_per_block % P.couple) return cudaErrorInvalidValue;
  // blocks needed to give every cell (every group) a warp (group of warps)
  const int64_t units = (C.n_cells + P.couple - 1) / P.couple, per_block = P.warps_per_block / P.couple;
  const int64_t need = (units + per_block - 1) / per_block;
  int blocks;
  P.smem_bytes = 0;
  if (cfg.driver == CHEM_DRIVER_PERSISTENT) {
    const int natural = occupancy(M, cfg.lu_precision, cfg.driver, cfg.warps_per_block);
    int bps = cfg.blocks_per_sm > 0 ? cfg.blocks_per_sm : natural;
    if (bps < 1) bps = 1;
    // fewer resident blocks than fit: pad the blocks' shared memory so that
    // the block scheduler cannot stack more than bps of them on one SM
    if (bps < natural)
      P.smem_bytes = (long long)pad_smem_to_blocks((size_t)P.tab_bytes + (size_t)P.cell_bytes * P.warps_per_block, bps);
    blocks = n_sm * bps;
    if (blocks > need) blocks = (int)need;
  } else {
    blocks = (int)need;
  }
  const bool f32 = cfg.lu_precision == 32;
  const bool coupled = cfg.couple > 1;      // warps_per_block is then the group size
  if (staged)
    return f32 ? launch_ks<float, true>(M, C, P, blocks, coupled, stream) : launch_ks<double, true>(M, C, P, blocks, coupled, stream);
  return f32 ? launch_ks<float, false>(M, C, P, blocks, coupled, stream) : launch_ks<double, false>(M, C, P, blocks, coupled, stream);
}

cudaError_t launch_adjoint(const MechDev &M, const CellsDev &C, const AdjDev &A, cudaStream_t stream) {
  if (C.n_cells <= 0) return cudaSuccess;
  SolveParams P{};
  // the forward's Wd and WL, the adjoint's arrays, then the partials dr_j/dy_l (at a_PP)
  P.wd_pad = (M.Wd_len + 1) & ~1;
  P.cell_bytes = (int)(((size_t)(M.a_PP + M.n_pairs) * sizeof(double) + 15) & ~(size_t)15);
  P.prec = 0;
  P.tab_bytes = 0;
  cudaError_t e = cudaSuccess;
  switch ((M.S + WARP - 1) / WARP) {
    case 1: e = launch_adj_t<1>(M, C, A, P, stream); break;
    case 2: e = launch_adj_t<2>(M, C, A, P, stream); break;
    case 3: e = launch_adj_t<3>(M, C, A, P, stream); break;
    case 4: e = launch_adj_t<4>(M, C, A, P, stream); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  theta_reduce_kernel<<<(M.R + 127) / 128, 128, 0, stream>>>(A.gcell, C.n_cells, M.R, A.dLdtheta, A.accumulate);
  return cudaGetLastError();
}

cudaError_t launch_count_flags(const int *flag, int64_t n, unsigned long long *acc, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  count_flags_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(flag, n, acc);
  return cudaGetLastError();
}

cudaError_t launch_tangent(const MechDev &M, const CellsDev &C, const TanDev &A, cudaStream_t stream) {
  if (C.n_cells <= 0) return cudaSuccess;
  SolveParams P{};
  // the tangent walk uses the forward's Wd and WL and one species vector after
  // them (the direction v at a_MU), not the adjoint's other arrays
  P.wd_pad = (M.Wd_len + 1) & ~1;
  P.cell_bytes = (int)(((size_t)(M.a_MU + M.S) * sizeof(double) + 15) & ~(size_t)15);
  P.prec = 0;
  switch ((M.S + WARP - 1) / WARP) {
    case 1: return launch_tan_t<1>(M, C, A, P, stream);
    case 2: return launch_tan_t<2>(M, C, A, P, stream);
    case 3: return launch_tan_t<3>(M, C, A, P, stream);
    case 4: return launch_tan_t<4>(M, C, A, P, stream);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_deriv_gather(const MechDev &M, const CellsDev &C, const double *kt, const double *y, double *f,
                                cudaStream_t stream) {
  if (C.n_cells <= 0) return cudaSuccess;
  const int cell_doubles = (M.Wd_len + 1) & ~1;
  const size_t smem = (size_t)M.tab.staged + (size_t)cell_doubles * sizeof(double) * GATHER_CELLS;
  cudaError_t e;
  const unsigned blocks = (unsigned)((C.n_cells + GATHER_CELLS - 1) / GATHER_CELLS);
  switch ((M.S + WARP - 1) / WARP) {
#define CHEM_GATHER_CASE(K_)                                                                                      \
    case K_:                                                                                                      \
      if ((e = allow_max_smem<deriv_gather_kernel<K_>>()) != cudaSuccess) return e;                          \
      deriv_gather_kernel<K_><<<blocks, GATHER_CELLS * WARP, smem, stream>>>(M, C.n_cells, kt, y, f, cell_doubles); \
      break;
    CHEM_GATHER_CASE(1) CHEM_GATHER_CASE(2) CHEM_GATHER_CASE(3) CHEM_GATHER_CASE(4)
#undef CHEM_GATHER_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_order_groups(const CellsDev &C, int G, int *bucket, int *hist, int *order, cudaStream_t stream) {
  if (C.n_cells <= 0 || G < 1) return cudaSuccess;
  const int64_t ng = (C.n_cells + G - 1) / G;
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int) * ORDER_BUCKETS, stream);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((ng + 255) / 256);
  order_group_keys_kernel<<<blocks, 256, 0, stream>>>(C, G, ng, bucket, hist);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  order_scan_kernel<<<1, 32, 0, stream>>>(hist);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  order_scatter_kernel<<<blocks, 256, 0, stream>>>(bucket, hist, order, ng);
  return cudaGetLastError();
}

cudaError_t launch_order_tape(const CellsDev &C, int *bucket, int *hist, int *order, cudaStream_t stream) {
  if (C.n_cells <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int) * ORDER_BUCKETS, stream);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((C.n_cells + 255) / 256);
  order_tape_keys_kernel<<<blocks, 256, 0, stream>>>(C, bucket, hist);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  order_scan_kernel<<<1, 32, 0, stream>>>(hist);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  order_scatter_kernel<<<blocks, 256, 0, stream>>>(bucket, hist, order, C.n_cells);
  return cudaGetLastError();
}

cudaError_t launch_order(const MechDev &M, const CellsDev &C, double rtol, double atol, int *bucket, int *hist,
                         int *order, cudaStream_t stream) {
  if (C.n_cells <= 0) return cudaSuccess;
  SolveParams P{};
  P.rtol = rtol;
  P.atol = atol;
  P.wd_pad = (M.Wd_len + 1) & ~1;
  P.cell_bytes = (int)(((size_t)P.wd_pad * sizeof(double) + 15) & ~(size_t)15);
  P.warps_per_block = ORDER_WARPS;
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int) * ORDER_HIST_INTS, stream);
  if (e != cudaSuccess) return e;
  switch ((M.S + WARP - 1) / WARP) {
    case 1: e = launch_order_t<1>(M, C, P, bucket, hist, stream); break;
    case 2: e = launch_order_t<2>(M, C, P, bucket, hist, stream); break;
    case 3: e = launch_order_t<3>(M, C, P, bucket, hist, stream); break;
    case 4: e = launch_order_t<4>(M, C, P, bucket, hist, stream); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  order_bucket_kernel<<<(unsigned)((C.n_cells + 255) / 256), 256, 0, stream>>>(bucket, hist, C.n_cells);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  order_scan_kernel<<<1, 32, 0, stream>>>(hist);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  order_scatter_kernel<<<(unsigned)((C.n_cells + 255) / 256), 256, 0, stream>>>(bucket, hist, order, C.n_cells);
  return cudaGetLastError();
}

}  // namespace chemgpu
