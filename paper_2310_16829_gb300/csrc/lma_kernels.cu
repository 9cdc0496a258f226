// CUDA kernels of the LMA hot path for sm_103a (GB300).
//
//   k_potential      step a1: v_s(x) = sum of Gaussian-sum atom potentials, t_s = exp(i sigma v_s)
//                    (Sec. 3.2, transmission function)
//   k_slice          step a3: multislice of each lattice translate u_i on its W x W window,
//                    transmit -> 2D FFT -> propagator and bandlimit -> inverse 2D FFT per slice
//                    (Fig. multislice_pseudocode on the window of option (ii), Sec. 4.2.1)
//   k_synth_detect   steps a4-a6: Psi_p = sum_j alpha_j U_{i_j} on the D x D probe window
//                    (Sec. 4.2.2), |DFT(Psi_p)|^2 summed over the annular detector (Sec. 3.1),
//                    FP64 accumulation over frozen-phonon configurations
//   k_finalize       step a6: average over configurations
//
// The 128 x 128 complex64 wave of one translate stays in registers of one
// 512-thread CTA for all slices (32 values per thread). The 2D DFT is split
// into three register passes over the 14 index bits (x = 4 n1 + r,
// y = 32 n1y + n2y, Cooley-Tukey with 128 = 32 * 4 on each axis):
//   pass A: 32-point DFT over n1 (x axis)                          thread (y, r)
//   pass B: 4-point DFTs over r (x axis, with pass A's twiddle W_128^(r k1),
//           none for r = 0) and n1y (y axis) + twiddle W_128^(n2y k1y)   group (k1, n2y)
//   pass C: 32-point DFT over n2y (y axis)                         thread (kx, k1y)
//           (kx permuted so that one warp of four holds only columns outside
//           the 2/3 bandlimit and skips the pass)
// The propagator multiply sits in pass C; the inverse runs the passes back
// (C, B, A) with conjugate twiddles, so no index permutation is ever stored.
// Between passes the data crosses threads through one shared table in which
// every thread writes only the entries it has just read (four barriers per
// slice); each warp stages the transmission rows it multiplies into its own
// table rows with cp.async while its inverse pass A runs. The transmission is
// stored with a periodic halo of W pixels ([ny + W][nx + W] per slice), so
// that every window is a plain rectangle of the array.
#include "lma_device.h"

#include <cuda_fp16.h>

#include <cstdio>
#include <cstring>
#include <vector>
#include <mutex>
#include <type_traits>

namespace lma_dev {

// exp(-2 pi i m / 128), m = 0..127: built on the host in FP64 and rounded once.
__constant__ float2 c_w128[128];
// W_32^M = (cos th, -sin th), th = 2 pi M / 32, as a scale times (1, ratio) or (ratio, 1):
// (cos th, tan th) where |cos th| >= |sin th| (M <= 4 or M >= 12), else (sin th, cot th);
// built on the host in FP64 and rounded once. |ratio| <= 1 in both forms.
__constant__ float2 c_tw32t[16];
// Pass-A twiddles of the slice kernel's pass B, tau_r = W_128^(r k1), r = 1..3, per k1 < 32,
// as a scale s_r times (1, t_r) for k1 < 16 and (t_r, 1) for k1 >= 16 (tangent form; the
// form is the same across a half-warp): c_twrA[k1] = (t1, s1, t2, s2), c_twrB[k1] = (t3,
// s3, s3 / s1, 0). Built on the host in FP64 and rounded once.
__constant__ float4 c_twrA[32];
__constant__ float4 c_twrB[32];

// ------------------------------------------------------------------------------------------
// complex helpers
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// the same sums as one packed FP32 instruction each (add.rn.f32x2, and fma.rn.f32x2 with -1,
// whose product is exact): bit for bit equal to cadd / csub, half the issued instructions
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cfma(float2 acc, float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}

// cfma with the coefficient given as (a.x, a.x, -a.y, a.y): the same four FMAs in the same
// order, as two packed FP32 instructions
__device__ __forceinline__ float2 cfma2(float2 acc, float4 a, float2 b) {
  return __ffma2_rn(make_float2(a.x, a.y), b, __ffma2_rn(make_float2(a.z, a.w), make_float2(b.y, b.x), acc));
}

__host__ __device__ constexpr int brev5(int k) {
  return ((k & 1) << 4) | ((k & 2) << 2) | (k & 4) | ((k & 8) >> 2) | ((k & 16) >> 4);
}


// Column kx of pass-C thread T (k1y = T >> 7). Logical warps 1 and 2 of each k1y group
// exchange their lanes l < 11, so that logical warp 1 holds kx = 43..74: with the 2/3
// bandlimit (|kx| <= 42 at W = 128) every one of its columns is masked and it skips
// pass C. The logical warps are rotated by k1y within the group, so that the four
// skipping warps have four different warp ids mod 4 (one per SM sub-partition). Every
// warp keeps 32 distinct kx mod 32 (conflict-free X2 accesses).
__device__ __forceinline__ int c_column(int T) {
  const int k1y = T >> 7;
  const int w = (((T >> 5) & 3) - k1y) & 3, l = T & 31;
  if (w == 1) return l < 11 ? 64 + l : 32 + l;
  if (w == 2) return l < 11 ? 32 + l : 64 + l;
  return 32 * w + l;
}

// compile-time loop: f(std::integral_constant<int, I>) for I = B..E-1
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// One radix-2 decimation-in-time butterfly on t[I] (a) and t[I + H] (b) with the
// twiddle W_32^M. A general twiddle w = s (1, t) or s (t, 1) with |t| <= 1 (the
// tangent form of an FMA butterfly) computes (u, v) = w b / s with two FMAs and
// X = a + s (u, v), Y = a - s (u, v) with four: two roundings per component, as for
// a plain complex product (Y is not formed as 2a - X, which would carry X's rounding
// error into Y).
// NX / NY: whether X = t[I] / Y = t[I + H] is needed; Z (M = 0 only): 1 if a is known to
// be zero, 2 if b is (the outputs are then copies of the other input, exactly as the sum
// and difference would give).
template <bool INV, int I, int H, int M, bool NX = true, bool NY = true, int Z = 0, int N = 32>
__device__ __forceinline__ void bfly(float2 (&t)[N]) {
  const float2 a = t[I];
  const float2 b = t[I + H];
  if constexpr (Z == 1) {
    static_assert(M == 0, "zero inputs are pruned in the first stage only");
    t[I] = b;
    t[I + H] = make_float2(-b.x, -b.y);
  } else if constexpr (Z == 2) {
    static_assert(M == 0, "zero inputs are pruned in the first stage only");
    t[I + H] = a;
  } else if constexpr (M == 0) {
    if constexpr (NX) t[I] = padd(a, b);
    if constexpr (NY) t[I + H] = psub(a, b);
  } else if constexpr (M == 8) {
    // w b = -i b (forward) or i b (inverse)
    const float2 wb = INV ? make_float2(-b.y, b.x) : make_float2(b.y, -b.x);
    if constexpr (NX) t[I] = cadd(a, wb);
    if constexpr (NY) t[I + H] = csub(a, wb);
  } else if constexpr (M == 4 || M == 12) {
    // w = (c, s) with |c| = |s| = r = 1/sqrt(2): w b = (c b.x - s b.y, c b.y + s b.x) is
    // r times a sum or difference of b.x and b.y, so X and Y take one add and one FMA
    // per component (two roundings, as for a general twiddle)
    const float r = c_w128[16].x;                       // cos(pi / 4), rounded once
    constexpr int sc = M == 4 ? 1 : -1;                 // sign of c
    constexpr int ss = INV ? 1 : -1;                    // sign of s: -r forward, +r inverse
    float u, v;                                         // w b = sc r (u, v)
    if constexpr (sc == ss) {
      u = b.x - b.y;
      v = b.y + b.x;
    } else {
      u = b.x + b.y;
      v = b.y - b.x;
    }
    const float rs = sc > 0 ? r : -r;
    if constexpr (NX) t[I] = make_float2(fmaf(rs, u, a.x), fmaf(rs, v, a.y));
    if constexpr (NY) t[I + H] = make_float2(fmaf(-rs, u, a.x), fmaf(-rs, v, a.y));
  } else if constexpr (M < 4 || M > 12) {
    // |cos| > |sin|: w b = cos th (b + i t b) with t = wy / wx (-tan th forward, +tan th
    // inverse): two FMAs form (u, v) = b + i t b, four more give X and Y
    const float2 k = c_tw32t[M];
    const float tq = INV ? k.y : -k.y;
    const float u = fmaf(-tq, b.y, b.x), v = fmaf(tq, b.x, b.y);
    if constexpr (NX) t[I] = make_float2(fmaf(k.x, u, a.x), fmaf(k.x, v, a.y));
    if constexpr (NY) t[I + H] = make_float2(fmaf(-k.x, u, a.x), fmaf(-k.x, v, a.y));
  } else {
    // |sin| > |cos|: w b = wy (c b + i b) with c = wx / wy, wy = -sin th forward, +sin th
    // inverse
    const float2 k = c_tw32t[M];
    const float sy = INV ? k.x : -k.x, ct = INV ? k.y : -k.y;
    const float u = fmaf(ct, b.x, -b.y), v = fmaf(ct, b.y, b.x);
    if constexpr (NX) t[I] = make_float2(fmaf(sy, u, a.x), fmaf(sy, v, a.y));
    if constexpr (NY) t[I + H] = make_float2(fmaf(-sy, u, a.x), fmaf(-sy, v, a.y));
  }
}

// In-register 32-point DFT, natural order in and out: radix-2 decimation in
// time on the bit-reversed input (a register renaming), 5 stages of spans 1..16.
// ZMODE 1: outputs 11..20 are not needed (the last stage skips them); ZMODE 2: inputs
// 11..20 are zero (the first stage copies instead of adding). Both hold for the pass-C
// columns of the slice kernel when the bandlimit radius is below 44: ky = k1y + 4 j has
// |ky| >= 44 for every j in 11..20.
__host__ __device__ constexpr bool in_gap(int j) { return j >= 11 && j <= 20; }
template <bool INV, int ZMODE = 0>
__device__ __forceinline__ void dft32(float2 (&v)[32]) {
  float2 t[32];
  static_for<0, 32>([&](auto k) {
    constexpr int K = decltype(k)::value;
    t[K] = v[brev5(K)];
  });
  static_for<0, 5>([&](auto st) {
    constexpr int H = 1 << decltype(st)::value;
    static_for<0, 16 / H>([&](auto blk) {
      static_for<0, H>([&](auto j) {
        constexpr int I = decltype(blk)::value * 2 * H + decltype(j)::value;
        constexpr int M = decltype(j)::value * (16 / H);
        // first stage: t[I] = v[brev5(I)], t[I + 1] = v[brev5(I) + 16]
        constexpr int Z = (ZMODE == 2 && H == 1) ? (in_gap(brev5(I)) ? 1 : (in_gap(brev5(I) + 16) ? 2 : 0)) : 0;
        constexpr bool NX = !(ZMODE == 1 && H == 16 && in_gap(I));
        constexpr bool NY = !(ZMODE == 1 && H == 16 && in_gap(I + 16));
        bfly<INV, I, H, M, NX, NY, Z>(t);
      });
    });
  });
  static_for<0, 32>([&](auto k) {
    constexpr int K = decltype(k)::value;
    v[K] = t[K];
  });
}

// In-register 16-point DFT, natural order in and out: the first four stages of dft32 on 16
// values (W_16^m = W_32^(2m), so stage H takes the twiddle index j (16 / H) of dft32)
__host__ __device__ constexpr int brev4(int k) { return ((k & 1) << 3) | ((k & 2) << 1) | ((k & 4) >> 1) | ((k & 8) >> 3); }
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&v)[16]) {
  float2 t[16];
  static_for<0, 16>([&](auto k) {
    constexpr int K = decltype(k)::value;
    t[K] = v[brev4(K)];
  });
  static_for<0, 4>([&](auto st) {
    constexpr int H = 1 << decltype(st)::value;
    static_for<0, 8 / H>([&](auto blk) {
      static_for<0, H>([&](auto j) {
        constexpr int I = decltype(blk)::value * 2 * H + decltype(j)::value;
        constexpr int M = decltype(j)::value * (16 / H);
        bfly<INV, I, H, M>(t);
      });
    });
  });
  static_for<0, 16>([&](auto k) {
    constexpr int K = decltype(k)::value;
    v[K] = t[K];
  });
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 s02 = padd(a0, a2), d02 = psub(a0, a2), s13 = padd(a1, a3), d13 = psub(a1, a3);
  // forward: X1 = d02 - i d13, X3 = d02 + i d13; inverse swaps the sign of i
  const float2 j13 = INV ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);
  a0 = padd(s02, s13);
  a2 = psub(s02, s13);
  a1 = padd(d02, j13);
  a3 = psub(d02, j13);
}

// dft4 with input Z known to be zero (Z = -1: none); the outputs are those of dft4
template <bool INV, int Z>
__device__ __forceinline__ void dft4z(float2& a0, float2& a1, float2& a2, float2& a3) {
  float2 s02, d02, s13, d13;
  if constexpr (Z == 2) {
    s02 = a0;
    d02 = a0;
  } else {
    s02 = cadd(a0, a2);
    d02 = csub(a0, a2);
  }
  if constexpr (Z == 1) {
    s13 = a3;
    d13 = make_float2(-a3.x, -a3.y);
  } else {
    s13 = cadd(a1, a3);
    d13 = csub(a1, a3);
  }
  const float2 j13 = INV ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, j13);
  a3 = csub(d02, j13);
}

// ------------------------------------------------------------------------------------------
// the three passes
// ------------------------------------------------------------------------------------------
// pass A, thread (y, r): v[n1] = psi(y, 4 n1 + r) -> v[k1] after the x-axis 32-point stage
// twA points at the row W_128^(r k), k = 0..31, of this thread's r; rows are 34
// entries apart so that the four r of a warp read distinct banks, two entries
// per 128-bit load
__device__ __forceinline__ void passA_fwd(float2 (&v)[32], const float2* twA) {
  dft32<false>(v);
  const float4* w4 = reinterpret_cast<const float4*>(twA);
#pragma unroll
  for (int k = 0; k < 32; k += 2) {
    const float4 w = w4[k / 2];
    if (k > 0) v[k] = cmul(v[k], make_float2(w.x, w.y));
    v[k + 1] = cmul(v[k + 1], make_float2(w.z, w.w));
  }
}

// pass B, group (k1, n2y): a[n1y * 4 + r] -> a[k1y * 4 + k2x]
// twB points at W_128^(n2y k1y), k1y = 0..3, of this group's n2y
__device__ __forceinline__ void passB_fwd(float2 (&a)[16], const float2* twB) {
#pragma unroll
  for (int q = 0; q < 4; ++q) dft4<false>(a[q * 4 + 0], a[q * 4 + 1], a[q * 4 + 2], a[q * 4 + 3]);
#pragma unroll
  for (int q = 0; q < 4; ++q) dft4<false>(a[0 * 4 + q], a[1 * 4 + q], a[2 * 4 + q], a[3 * 4 + q]);
#pragma unroll
  for (int k1y = 1; k1y < 4; ++k1y) {
    const float2 w = twB[k1y];
#pragma unroll
    for (int q = 0; q < 4; ++q) a[k1y * 4 + q] = cmul(a[k1y * 4 + q], w);
  }
}

// pass B of the slice kernel with pass A's twiddles W_128^(r k1) moved into it: r is
// this thread's own index here, so r = 0 needs none (24 products per thread instead of
// 31). Forward, they are fused into the radix-4 stage over r: with (u_r, v_r) = tau_r a_r
// / s_r (two FMAs each) and rho = s3 / s1,
//   a0 + tau_2 a2 = a0 + s2 (u2, v2),   tau_1 a1 + tau_3 a3 = s1 ((u1, v1) + rho (u3, v3)),
// 22 instructions per radix-4 stage against 28 for three products and the plain stage.
// COT selects the form of the twiddles (k1 >= 16).
template <bool COT>
__device__ __forceinline__ void tw_uv(float2 a, float t, float& u, float& v) {
  if constexpr (COT) {
    u = fmaf(t, a.x, -a.y);
    v = fmaf(t, a.y, a.x);
  } else {
    u = fmaf(-t, a.y, a.x);
    v = fmaf(t, a.x, a.y);
  }
}
template <bool COT, int SKIP = -1>
__device__ __forceinline__ void dft4_tw(float2& a0, float2& a1, float2& a2, float2& a3, const float4 kA,
                                        const float4 kB) {
  float u1, v1, u2, v2, u3, v3;
  tw_uv<COT>(a1, kA.x, u1, v1);
  tw_uv<COT>(a2, kA.z, u2, v2);
  tw_uv<COT>(a3, kB.x, u3, v3);
  const float s1 = kA.y, s2 = kA.w, rho = kB.z;
  const float2 s02 = make_float2(fmaf(s2, u2, a0.x), fmaf(s2, v2, a0.y));
  const float2 d02 = make_float2(fmaf(-s2, u2, a0.x), fmaf(-s2, v2, a0.y));
  const float2 P = make_float2(fmaf(rho, u3, u1), fmaf(rho, v3, v1));    // (tau_1 a1 + tau_3 a3) / s1
  const float2 D = make_float2(fmaf(-rho, u3, u1), fmaf(-rho, v3, v1));  // (tau_1 a1 - tau_3 a3) / s1
  // forward: X1 = d02 - i d13, X3 = d02 + i d13
  // output SKIP is not needed
  if constexpr (SKIP != 0) a0 = make_float2(fmaf(s1, P.x, s02.x), fmaf(s1, P.y, s02.y));
  if constexpr (SKIP != 2) a2 = make_float2(fmaf(-s1, P.x, s02.x), fmaf(-s1, P.y, s02.y));
  if constexpr (SKIP != 1) a1 = make_float2(fmaf(s1, D.y, d02.x), fmaf(-s1, D.x, d02.y));
  if constexpr (SKIP != 3) a3 = make_float2(fmaf(-s1, D.y, d02.x), fmaf(s1, D.x, d02.y));
}
// a * conj(tau) for tau = s (1, t) or s (t, 1)
template <bool COT>
__device__ __forceinline__ float2 tw_conj(float2 a, float s, float t) {
  float u, v;
  if constexpr (COT) {
    u = fmaf(t, a.x, a.y);
    v = fmaf(t, a.y, -a.x);
  } else {
    u = fmaf(t, a.y, a.x);
    v = fmaf(-t, a.x, a.y);
  }
  return make_float2(s * u, s * v);
}
// With PRUNE, column k2x = MC of this half lies outside the bandlimit for every ky
// (k1 < 16: kx = k1 + 64, |kx| >= 49; k1 >= 16: kx = k1 + 32 >= 48; the radius is below
// 44): forward it is not formed, inverse it is zero (C writes zeros there).
template <bool COT, bool PRUNE>
__host__ __device__ constexpr int masked_k2x() { return PRUNE ? (COT ? 1 : 2) : -1; }
template <bool COT, bool PRUNE>
__device__ __forceinline__ void passB_fwd_tw(float2 (&a)[16], const float2* twB, const float4 kA, const float4 kB) {
  constexpr int MC = masked_k2x<COT, PRUNE>();
#pragma unroll
  for (int q = 0; q < 4; ++q) dft4_tw<COT, MC>(a[q * 4 + 0], a[q * 4 + 1], a[q * 4 + 2], a[q * 4 + 3], kA, kB);
  static_for<0, 4>([&](auto qq) {
    constexpr int q = decltype(qq)::value;
    if constexpr (q != MC) dft4<false>(a[0 * 4 + q], a[1 * 4 + q], a[2 * 4 + q], a[3 * 4 + q]);
  });
#pragma unroll
  for (int k1y = 1; k1y < 4; ++k1y) {
    const float2 w = twB[k1y];
    static_for<0, 4>([&](auto qq) {
      constexpr int q = decltype(qq)::value;
      if constexpr (q != MC) a[k1y * 4 + q] = cmul(a[k1y * 4 + q], w);
    });
  }
}
template <bool COT, bool PRUNE>
__device__ __forceinline__ void passB_inv_tw(float2 (&a)[16], const float2* twB, const float4 kA, const float4 kB) {
  constexpr int MC = masked_k2x<COT, PRUNE>();
#pragma unroll
  for (int k1y = 1; k1y < 4; ++k1y) {
    const float2 w = twB[k1y];
    static_for<0, 4>([&](auto qq) {
      constexpr int q = decltype(qq)::value;
      if constexpr (q != MC) a[k1y * 4 + q] = cmulc(a[k1y * 4 + q], w);
    });
  }
  static_for<0, 4>([&](auto qq) {
    constexpr int q = decltype(qq)::value;
    if constexpr (q != MC) dft4<true>(a[0 * 4 + q], a[1 * 4 + q], a[2 * 4 + q], a[3 * 4 + q]);
  });
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    dft4z<true, MC>(a[q * 4 + 0], a[q * 4 + 1], a[q * 4 + 2], a[q * 4 + 3]);
    a[q * 4 + 1] = tw_conj<COT>(a[q * 4 + 1], kA.y, kA.x);
    a[q * 4 + 2] = tw_conj<COT>(a[q * 4 + 2], kA.w, kA.z);
    a[q * 4 + 3] = tw_conj<COT>(a[q * 4 + 3], kB.y, kB.x);
  }
}

// shared-memory layouts of the synthesis kernel's exchanges (float2 units); row
// paddings keep the 64-bit accesses of every half-warp on 16 distinct bank pairs and
// make every address a per-thread base plus a compile-time offset
//   X1 (A -> B), 512 x 34 entries: element (y, r, k1) at TA*34 + k1, TA = 4y + r
//      (A writes two entries per 128-bit store: 8 lanes on 8 distinct 16-byte slots)
//   X2 (B -> C), 16384 entries: element (k1y, k2x, n2y, k1x) at ((k1y*4 + k2x)*32 + n2y)*32 + k1x
constexpr int kX1 = 512 * 34;

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ------------------------------------------------------------------------------------------
// per-CTA shared tables
// ------------------------------------------------------------------------------------------
// twA[r*34 + k] = W_128^(r k) (k < 32); twB[n2y*4 + k1y] = W_128^(n2y k1y)
constexpr int kTwA = 4 * 34;
__device__ __forceinline__ void load_twiddles(float2* twA, float2* twB, int T) {
  if (T < 128) {
    twA[(T >> 5) * 34 + (T & 31)] = c_w128[((T >> 5) * (T & 31)) & 127];
    twB[T] = c_w128[((T >> 2) * (T & 3)) & 127];
  }
}

// ------------------------------------------------------------------------------------------
// step a3: slice kernel
// ------------------------------------------------------------------------------------------
// The slice kernel keeps every exchange in one table of 512 rows x 34 entries (row TA =
// 4 y + r, entry k), and every thread writes only the entries it has just read:
//   A thread (y, r):   row TA = T, entries 0..31: its pass-A outputs k1 (X1), later its
//                      pass-B-inverse inputs (X4)
//   B thread (k1, n2y): entries k1 of rows 4 (32 q + n2y) + r, q, r < 4: X1 element
//                      (y = 32 q + n2y, r, k1) at slot (q, r); its pass-B output (k1y, k2x)
//                      goes to slot (q, r) = (k2x, k1y) (X2) and its inverse output
//                      (q, r) back to slot (q, r) (X4)
//   C thread (kx, k1y): entry k1x of rows 4 (32 k2x + j) + k1y, j < 32 (read, write back)
//   warp w:            rows 32 w .. 32 w + 31 (1056 entries) also hold the transmission
//                      of its 8 window rows y = 8 w .. 8 w + 7 as 8 rows of 132 entries
// No entry is written by one thread while another thread of the CTA may still read it,
// so the only CTA barriers are the four that publish a phase's writes (read-after-write);
// the transmission is shared within a warp only (__syncwarp). With rows of 34 entries the
// A side moves entry pairs (k, k + 1) with 128-bit accesses, a quarter-warp's 8 rows on 8
// distinct 16-byte slots (17 TA + k/2 mod 8); the 64-bit B and C accesses of a half-warp
// are 16 consecutive entries of one row (of two rows 128 x 34 entries apart in the warps
// that mix k2x), on 16 distinct bank pairs.
constexpr int kXP = 34;
constexpr int kXRows = 512 * kXP;
constexpr int kTRow = 132;   // staged transmission row: 4 table rows
static_assert(8 * kTRow <= 32 * kXP, "a warp's 8 transmission rows fit its 32 table rows");
// propagator table P[a * 65 + b] = e_x(a) e_y(b) for |kx| = a, |ky| = b <= 64, zero
// outside the bandlimit (e_x and e_y depend on k^2 only); the odd row length spreads
// the 16 consecutive a of a half-warp over distinct bank pairs
constexpr int kPRow = 65;
constexpr int kPTab = kPRow * kPRow;
constexpr int kSliceSmemFloat2 = kXRows + 128 + 128 + kPTab;

// Warp w copies window rows 8 w .. 8 w + 7 of one slice (g points at the first) into its
// table rows (asynchronous; the warp's threads read them after cp_async_wait_all and
// __syncwarp). With an even window origin in 16-byte pieces, 512 contiguous bytes per
// instruction; with an odd origin in 8-byte pieces.
template <bool EVEN>
__device__ __forceinline__ void stage_t_warp(float2* region, const float2* g, int pitch, int lane) {
  if (EVEN) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int yl = i >> 1, x = 64 * (i & 1) + 2 * lane;
      cp_async16(region + yl * kTRow + x, g + static_cast<size_t>(yl) * pitch + x);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const int yl = i >> 2, x = 32 * (i & 3) + lane;
      cp_async8(region + yl * kTRow + x, g + static_cast<size_t>(yl) * pitch + x);
    }
  }
  cp_async_commit();
}

// One translate per CTA at a time, items taken as SliceLaunch's mode says; EVEN selects
// the window-origin parity of the translates in the list; HALF writes the exit wave as
// FP16 pairs scaled by a per-wave power of two; PRUNE (every job's bandlimit radius below
// 44 pixels) skips the spectral entries that the bandlimit zeroes for every column (pass
// B's masked k2x column per half, pass C's entries 11..20), with the same results.
template <bool EVEN, bool HALF, bool PRUNE>
__global__ void __launch_bounds__(kThreads, 1) k_slice(const SliceLaunch a, const int mode) {
  extern __shared__ __align__(16) float2 sm[];
  float2* X = sm;              // exchange table, 512 rows x kXP
  float4* twr = reinterpret_cast<float4*>(X + kXRows);   // [0, 32): c_twrA, [32, 64): c_twrB
  float2* twB = X + kXRows + 128;
  float2* ptab = twB + 128;    // propagator table, kPRow x kPRow

  const int T = threadIdx.x;
  if (T < 128) twB[T] = c_w128[((T >> 2) * (T & 3)) & 127];
  if (T < 64) twr[T] = T < 32 ? c_twrA[T] : c_twrB[T - 32];
  // A layout: thread (y, r), TA = T
  const int ya = T >> 2, ra = T & 3;
  // B layout: groups (k1 = (T & 15) + 16 h, n2y = T >> 4), h = 0, 1
  const int k1lo = T & 15, n2y = T >> 4;
  // C layout: thread (kx, k1y), kx permuted within each k1y group (c_column)
  const int kx = c_column(T), k1y = T >> 7, k1x = kx & 31, k2x = kx >> 5;
  const float2* tB = twB + n2y * 4;
  const int kxs = kx < 64 ? kx : kx - 128;
  // entry j of this C thread: ky = k1y + 4 j, |ky| = k1y + 4 j (j < 16), 128 - k1y - 4 j
  const float2* const pp = ptab + (kxs < 0 ? -kxs : kxs) * kPRow + k1y;            // + 4 j
  const float2* const pm = ptab + (kxs < 0 ? -kxs : kxs) * kPRow + 128 - k1y;      // - 4 j
  bool c_live = false;
  int cur_job = -1;
  __shared__ int s_next;
  __shared__ int s_wmax;      // FP16 store: bits of the wave's largest |component| (order-preserving for >= 0)
  float2* const xa = X + T * kXP;                                 // A row, + n or k1
  float2* const xb = X + (4 * n2y) * kXP + k1lo;                  // B slot (q, r): + (128 q + r) * kXP, + 16 (h = 1)
  float2* const xc = X + (128 * k2x + k1y) * kXP + k1x;           // C entry j: + 4 j * kXP
  const int lane = T & 31;
  float2* const xw = X + (T >> 5) * (32 * kXP);                   // this warp's table rows
  const float2* const tr = xw + (ya & 7) * kTRow + ra;            // t(y, 4 n + r) at + 4 n

  __syncthreads();   // twiddles

  for (int it = 0;; ++it) {
    int li;
    if (mode == kSliceDynamic) {
      if (T == 0) s_next = atomicAdd(a.counter, 1);
      __syncthreads();   // the previous item ended with a barrier: s_next is free to rewrite
      li = s_next;
    } else {
      li = blockIdx.x + it * gridDim.x;
    }
    if (li >= a.n_list) break;
    if (HALF && T == 0) s_wmax = 0;   // the previous item's reads ended at its last barrier
    int jb = 0;
    while (jb + 1 < a.n_jobs && li >= a.start[jb + 1]) ++jb;
    const SliceJob& J = a.job[jb];
    if (jb != cur_job) {
      // the previous item's last barrier has passed: the table is free; the X1 barrier
      // below publishes it before pass C reads it
      cur_job = jb;
      for (int e = T; e < kPTab; e += kThreads) {
        const int pa = e / kPRow, pb = e - pa * kPRow;
        ptab[e] = pa * pa + pb * pb <= J.r2max ? cmul(J.ex[pa], J.ey[pb]) : make_float2(0.f, 0.f);
      }
      // a warp whose columns are all outside the bandlimit skips pass C: its spectrum is zero
      c_live = __any_sync(0xffffffffu, kxs * kxs <= J.r2max);
    }
    const int n_slices = J.n_slices;
    const int pitch = J.nx + kW;                                  // padded row
    const size_t slice_elems = static_cast<size_t>(pitch) * (J.ny + kW);
    const int item = a.list[li];
    const int cfg = item / J.n_translates;
    const int ti = item - cfg * J.n_translates;
    const int ia = ti % J.lat_nax, ib = ti / J.lat_nax;
    int ox = (J.lat_ox + ia * J.lat_sx - kW / 2) % J.nx;
    if (ox < 0) ox += J.nx;
    int oy = (J.lat_oy + ib * J.lat_sy - kW / 2) % J.ny;
    if (oy < 0) oy += J.ny;
    // the halo of W pixels keeps every window inside the padded array
    const float2* const gsrc = J.t + cfg * J.t_slot + static_cast<size_t>(oy + 8 * (T >> 5)) * pitch + ox;

    stage_t_warp<EVEN>(xw, gsrc, pitch, lane);
    float2 v[32];
#pragma unroll
    for (int n1 = 0; n1 < 32; ++n1) v[n1] = J.uW[ya * kW + 4 * n1 + ra];

    for (int s = 0; s < n_slices; ++s) {
      // transmission (Sec. 3.2): psi <- t_s psi, from the warp's staged rows
      cp_async_wait_all();
      __syncwarp();
#pragma unroll
      for (int n1 = 0; n1 < 32; ++n1) v[n1] = cmul(v[n1], tr[4 * n1]);

      // forward 2D DFT; X1 goes to this warp's rows once every lane has read its t
      dft32<false>(v);
      __syncwarp();
      float4* const xa4 = reinterpret_cast<float4*>(xa);
#pragma unroll
      for (int k = 0; k < 32; k += 2) xa4[k / 2] = make_float4(v[k].x, v[k].y, v[k + 1].x, v[k + 1].y);
      __syncthreads();
      float2 b0[16], b1[16];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          b0[q * 4 + r] = xb[(128 * q + r) * kXP];
          b1[q * 4 + r] = xb[(128 * q + r) * kXP + 16];
        }
      passB_fwd_tw<false, PRUNE>(b0, tB, twr[k1lo], twr[32 + k1lo]);
      passB_fwd_tw<true, PRUNE>(b1, tB, twr[16 + k1lo], twr[48 + k1lo]);
      // X2: element (k1y, k2x) to slot (q, r) = (k2x, k1y); a pruned column is not written
      // (pass C finds finite values of this slice's X1 there and multiplies them by zero)
      static_for<0, 4>([&](auto qq) {
        constexpr int q = decltype(qq)::value;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          if constexpr (q != masked_k2x<false, PRUNE>()) xb[(128 * q + r) * kXP] = b0[r * 4 + q];
          if constexpr (q != masked_k2x<true, PRUNE>()) xb[(128 * q + r) * kXP + 16] = b1[r * 4 + q];
        }
      });
      __syncthreads();
      if (c_live) {
        float2 c[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) c[j] = xc[j * 4 * kXP];
        dft32<false, PRUNE ? 1 : 0>(c);
        // propagation (Sec. 3.2): exp(-i pi lambda eps |k|^2), bandlimit, 1/W^2
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (!PRUNE || !in_gap(j)) c[j] = cmul(c[j], j < 16 ? pp[4 * j] : pm[-4 * j]);
        dft32<true, PRUNE ? 2 : 0>(c);
#pragma unroll
        for (int j = 0; j < 32; ++j) xc[j * 4 * kXP] = c[j];
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) xc[j * 4 * kXP] = make_float2(0.f, 0.f);
      }
      __syncthreads();
      static_for<0, 4>([&](auto qq) {
        constexpr int q = decltype(qq)::value;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          if constexpr (q != masked_k2x<false, PRUNE>()) b0[r * 4 + q] = xb[(128 * q + r) * kXP];
          if constexpr (q != masked_k2x<true, PRUNE>()) b1[r * 4 + q] = xb[(128 * q + r) * kXP + 16];
        }
      });
      passB_inv_tw<false, PRUNE>(b0, tB, twr[k1lo], twr[32 + k1lo]);
      passB_inv_tw<true, PRUNE>(b1, tB, twr[16 + k1lo], twr[48 + k1lo]);
      // X4: element (y = 32 q + n2y, r) back to slot (q, r)
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          xb[(128 * q + r) * kXP] = b0[q * 4 + r];
          xb[(128 * q + r) * kXP + 16] = b1[q * 4 + r];
        }
      __syncthreads();
      {
        const float4* const xa4 = reinterpret_cast<const float4*>(xa);
#pragma unroll
        for (int k = 0; k < 32; k += 2) {
          const float4 p = xa4[k / 2];
          v[k] = make_float2(p.x, p.y);
          v[k + 1] = make_float2(p.z, p.w);
        }
      }
      // the warp's rows are free again once every lane has read them: prefetch the next
      // slice's transmission while the inverse pass A runs
      __syncwarp();
      if (s + 1 < n_slices) stage_t_warp<EVEN>(xw, gsrc + (s + 1) * slice_elems, pitch, lane);
      dft32<true>(v);
    }

    if constexpr (HALF) {
      // power-of-two scale bringing the largest component into [0.5, 1): the scaling
      // is exact, the FP16 rounding (2^-11 of that component) is the only error
      float m = 0.f;
#pragma unroll
      for (int n1 = 0; n1 < 32; ++n1) m = fmaxf(m, fmaxf(fabsf(v[n1].x), fabsf(v[n1].y)));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if ((T & 31) == 0) atomicMax(&s_wmax, __float_as_int(m));
      __syncthreads();
      const float mx = __int_as_float(s_wmax);
      int e = 0;
      if (mx > 0.f) frexpf(mx, &e);
      const float sc = ldexpf(1.f, -e);
      const int oi = a.out_index ? a.out_index[li] : ti;
      // the warp's 8 rows go through its own table rows (rows of 132 pairs: the 4-byte
      // writes of 8 rows x 4 residues fall on 32 distinct banks) and out as 16-byte
      // stores, 512 contiguous bytes per instruction (the FP16 pairs of one thread are
      // 16 bytes apart in the wave, so direct stores would write half sectors)
      __half2* const hs = reinterpret_cast<__half2*>(xw);
#pragma unroll
      for (int n1 = 0; n1 < 32; ++n1) hs[(ya & 7) * 132 + 4 * n1 + ra] = __floats2half2_rn(v[n1].x * sc, v[n1].y * sc);
      __syncwarp();
      uint4* const dst = reinterpret_cast<uint4*>(static_cast<__half2*>(J.Uh) + cfg * J.u_slot +
                                                  static_cast<size_t>(oi) * (kW * kW) + (8 * (T >> 5)) * kW);
#pragma unroll
      for (int yl = 0; yl < 8; ++yl)
        dst[yl * (kW / 4) + lane] = *reinterpret_cast<const uint4*>(hs + yl * 132 + 4 * lane);
      if (T == 0) J.Uscale[static_cast<size_t>(cfg) * J.n_translates + oi] = ldexpf(1.f, e);
    } else {
      const int oi = a.out_index ? a.out_index[li] : ti;
      float2* ud = J.U + cfg * J.u_slot + static_cast<size_t>(oi) * (kW * kW) + ya * kW + ra;
#pragma unroll
      for (int n1 = 0; n1 < 32; ++n1) ud[4 * n1] = v[n1];
    }
    __syncthreads();  // the table, s_wmax and s_next are rewritten by the next item
  }
}

// ------------------------------------------------------------------------------------------
// step a3 with the 32-point DFT passes on the tensor cores (precision LMA_PREC_MIXED)
// ------------------------------------------------------------------------------------------
// Passes A and C of k_slice are 32-point DFTs of 512 rows of 32 complex values each (rows
// (y, r) in pass A, rows (kx, k1y) in pass C): as a product, Y = X F with F[n][k] = W_32^(n k),
// a [512 x 32] x [32 x 32] complex GEMM. In real form, row [Re x | Im x] (K = 64) times
// B = [[Re F, Im F], [-Im F, Re F]] (64 x 64) gives [Re y | Im y]. Each operand is split into
// FP16 parts, x = x_hi + x_lo (x_hi = fp16(x), x_lo = fp16(x - x_hi)), and the product is
// taken as x_lo F_hi + x_hi F_lo + x_hi F_hi with FP32 accumulation in tensor memory (the
// x_lo F_lo term, 2^-22 of the product, is dropped): tcgen05.mma kind::f16, M = 128 rows per
// tile, four tiles per pass. The inverse DFT (conj F) has its own B, [[Re F, -Im F], [Im F,
// Re F]] (Re y = Re x Re F + Im x Im F, Im y = -Re x Im F + Im x Re F). Pass B, the transmission
// and the propagator products stay on the CUDA cores in FP32, as in k_slice.
//
// Scale. FP16 holds 11 significant bits between 2^-14 and 65504. The wave enters with a
// power-of-two scale that brings its norm to (2^10, 2^11]; |t| = 1 and the bandlimited
// propagator has modulus <= 1, so the norm never grows. Every GEMM operand is bounded by
// the norm of its array: 2^11 before pass A, sqrt(512) 2^11 < 65504 before pass C, and with
// the propagator scaled by 2^-7 (instead of 2^-14 = 1/W^2) 2^11 before the inverse pass C
// and sqrt(512) 2^11 before the inverse pass A; the remaining 2^-7 is applied with the next
// transmission. Typical magnitudes (norm / 128) stay above 16, so the FP16 low parts are
// normal numbers almost everywhere.
//
// Shared memory: the A operand of tile t (rows 128 t .. 128 t + 127, FP16 high and low parts,
// 2 x 16 KiB) lies inside the exchange-table rows of the same 128 threads, which the pass-B
// exchanges use at other times; the forward and inverse B (high and low parts, 4 x 8 KiB)
// have their own space. Operands are
// K-major without swizzle: core matrices of 8 rows x 16 bytes, 128 bytes apart along K and
// 1024 bytes apart along the rows.
namespace tc {

constexpr uint32_t kTileBytes = 128 * kXP * 8;               // 128 table rows of kXP float2
static_assert(kTileBytes == 34816, "a tile's table rows");
constexpr uint32_t kHalfBytes = 16384;                        // one FP16 part of a 128 x 64 tile
constexpr int kTmemCols = 256;                                // 4 tiles x 64 FP32 columns
constexpr uint32_t kBBytes = 8192;                            // one FP16 part of B (64 x 64)
constexpr float kPropScale = 128.f;                           // 2^-7 / 2^-14: propagator factor
constexpr float kTransScale = 1.f / 128.f;                    // 2^-7 with each transmission

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// byte offset of element (row, k) in a no-swizzle K-major operand with K = 64 FP16
__host__ __device__ constexpr uint32_t op_offset(int row, int k) {
  return static_cast<uint32_t>((row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}
// shared-memory matrix descriptor: start, leading (K) byte offset 128, stride (row-group)
// byte offset 1024, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return static_cast<uint64_t>((saddr >> 4) & 0x3FFF) | (static_cast<uint64_t>(128 >> 4) << 16) |
         (static_cast<uint64_t>(1024 >> 4) << 32) | (static_cast<uint64_t>(1) << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator, FP16 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
  return (1u << 4) | (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}
__device__ __forceinline__ uint32_t try_wait(uint32_t mbar, uint32_t phase) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(mbar), "r"(phase)
      : "memory");
  return done;
}
// try_wait that lets the thread be suspended up to kSuspendNs while the phase is incomplete
// (woken when it completes), instead of spinning on the shared-memory pipe
constexpr uint32_t kSuspendNs = 1000000;
constexpr int kSuspendLimit = 2000;          // at least 2 s in all before giving up
__device__ __forceinline__ uint32_t try_wait_sleep(uint32_t mbar, uint32_t phase) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(mbar), "r"(phase), "r"(kSuspendNs)
      : "memory");
  return done;
}
// wait for the given phase of the mbarrier, giving up after kSuspendLimit suspended tries
// (one thread)
__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t phase) {
  uint32_t done = 0;
  for (int it = 0; it < kSuspendLimit && !done; ++it) done = try_wait_sleep(mbar, phase);
  return done != 0;
}
// the same for a whole warp: lane 0 polls, then every lane observes the completed phase
// itself (one try_wait each, for the memory ordering), so 31 lanes do not spin on the
// shared-memory pipe; warp-uniform result
__device__ __forceinline__ bool wait_phase_warp(uint32_t mbar, uint32_t phase) {
  uint32_t done = 0;
  if ((threadIdx.x & 31) == 0) done = wait_phase(mbar, phase) ? 1u : 0u;
  done = __shfl_sync(0xffffffffu, done, 0);
  if (done) done = try_wait(mbar, phase);
  return __all_sync(0xffffffffu, done != 0);
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// the 64 FP32 columns of this thread's TMEM lane from column c: y[k] = (col k, col 32 + k)
__device__ __forceinline__ void load_row(uint32_t taddr, float2 (&y)[32]) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,"
      "%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
        "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
        "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
        "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 32; ++k) y[k] = make_float2(__uint_as_float(r[k]), __uint_as_float(r[32 + k]));
}

// Row `row` of a tile's A operand from x: K index k < 32 holds Re x[k], k >= 32 Im x[k - 32];
// high parts to `hi`, low parts to `lo` (16-byte stores: a quarter-warp's 8 rows fill 128
// contiguous bytes)
__device__ __forceinline__ void store_row(unsigned char* hi, unsigned char* lo, const float2 (&x)[32], int row) {
  const uint32_t base = op_offset(row, 0);
#pragma unroll
  for (int kb = 0; kb < 8; ++kb) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int n = (kb & 3) * 8 + 2 * q;
      const float a = kb < 4 ? x[n].x : x[n].y;
      const float b = kb < 4 ? x[n + 1].x : x[n + 1].y;
      const __half2 hh = __floats2half2_rn(a, b);
      const float2 hf = __half22float2(hh);
      const __half2 ll = __floats2half2_rn(a - hf.x, b - hf.y);
      h[q] = *reinterpret_cast<const uint32_t*>(&hh);
      l[q] = *reinterpret_cast<const uint32_t*>(&ll);
    }
    *reinterpret_cast<uint4*>(hi + base + kb * 128) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(lo + base + kb * 128) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

// the MMAs of one pass over the four tiles: forward D = A B (N = 64), inverse by sub-blocks
// (N = 32); products lo x hi, hi x lo, hi x hi, the first overwriting D
// named barrier of the 128 threads of tile t (barrier 0 is __syncthreads)
__device__ __forceinline__ void tile_sync(int t) { asm volatile("bar.sync %0, 128;" ::"r"(t + 1) : "memory"); }

// the 12 MMAs of tile t of one pass: products lo x hi, hi x lo, hi x hi over four K steps of
// 16, the first overwriting D; forward or inverse B
template <bool INV>
__device__ __forceinline__ void issue_tile(uint32_t smA, uint32_t smB, uint32_t tmem, int t) {
  // descriptors differ only in their start-address field: base descriptor + (offset >> 4)
  // (every operand lies below 256 KiB, so the 14-bit field never carries)
  const uint64_t dB = sdesc(smB + (INV ? 2 * kBBytes : 0));
  const uint64_t aH = sdesc(smA + t * kTileBytes);
  constexpr uint64_t kLo = kHalfBytes >> 4, kBLo = kBBytes >> 4;
  const uint32_t d = tmem + 64 * t;
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const uint64_t a0 = p == 0 ? aH + kLo : aH;
    const uint64_t b0 = p == 1 ? dB + kBLo : dB;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
      mma(d, a0 + kk * 16, b0 + kk * 16, idesc(128, 64), (p > 0 || kk > 0) ? 1u : 0u);
  }
}

}  // namespace tc

// B operands of the forward and inverse 32-point DFT, high and low FP16 parts each, in the
// operand layout (built on the host in FP64: B^T[n][k], n the output column of [Re y | Im y],
// k the input of [Re x | Im x])
__device__ __align__(16) unsigned char g_tc_dft32[4 * tc::kBBytes];

constexpr int kSliceTcSmemBytes = kXRows * 8 + 4 * tc::kBBytes + 64 * 16 + 128 * 8 + kPTab * 8 + 4 * 8 + 16;

// One translate per CTA at a time (persistent CTAs, item li = blockIdx + k gridDim); the
// exit waves are complex64. status: set to 1 when a tensor-core wait gives up.
//
// The four M-tiles of a pass are independent: tile t is rows 128 t .. 128 t + 127, the rows
// of warps 4 t .. 4 t + 3, whose A operand lies in those threads' own table rows and whose
// accumulator is TMEM columns 64 t .. 64 t + 63. Each tile synchronizes its 128 threads with
// a named barrier, one elected thread issues the tile's MMAs and commits them to the tile's
// mbarrier, and the tile's threads read their rows back as soon as it completes: the tensor
// cores work on one tile while the CUDA cores split, store or read back the others. CTA
// barriers remain where data cross tiles: the pass-B exchanges (X1..X4), the reads of X2
// before pass C's operands overwrite the table, and the X3 writes after every tile's
// inverse pass C.
template <bool EVEN, bool PRUNE>
__global__ void __launch_bounds__(kThreads, 1) k_slice_tc(const SliceLaunch a, int* status) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  float2* X = reinterpret_cast<float2*>(smraw);                                   // exchange table
  unsigned char* const sB = smraw + kXRows * 8;                    // forward B hi, lo; inverse B hi, lo
  float4* twr = reinterpret_cast<float4*>(sB + 4 * tc::kBBytes);
  float2* twB = reinterpret_cast<float2*>(twr + 64);
  float2* ptab = twB + 128;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(ptab + kPTab);      // one per tile
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 4);

  const int T = threadIdx.x, warp = T >> 5, lane = T & 31;
  const int tile = T >> 7;
  const bool elected = (T & 127) == 0;
  if (T < 128) twB[T] = c_w128[((T >> 2) * (T & 3)) & 127];
  if (T < 64) twr[T] = T < 32 ? c_twrA[T] : c_twrB[T - 32];
  for (int i = T; i < 4 * static_cast<int>(tc::kBBytes) / 16; i += kThreads)
    reinterpret_cast<uint4*>(sB)[i] = reinterpret_cast<const uint4*>(g_tc_dft32)[i];
  if (T < 4) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(mbar + T)) : "memory");
  if (T == 0) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(tmem_slot)),
                 "r"(tc::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t mb = tc::smem_u32(mbar + tile);
  // this thread's TMEM lane: tile warp / 4, lane 32 (warp % 4) + lane = row T % 128
  const uint32_t t_row = tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + 64 * tile;
  const uint32_t smA = tc::smem_u32(smraw), smB = tc::smem_u32(sB);
  unsigned char* const aHi = smraw + tile * tc::kTileBytes;
  unsigned char* const aLo = aHi + tc::kHalfBytes;
  const int arow = T & 127;

  const int ya = T >> 2, ra = T & 3;
  const int k1lo = T & 15, n2y = T >> 4;
  const int kx = c_column(T), k1y = T >> 7, k1x = kx & 31, k2x = kx >> 5;
  const float2* tB = twB + n2y * 4;
  const int kxs = kx < 64 ? kx : kx - 128;
  const float2* const pp = ptab + (kxs < 0 ? -kxs : kxs) * kPRow + k1y;
  const float2* const pm = ptab + (kxs < 0 ? -kxs : kxs) * kPRow + 128 - k1y;
  bool c_live = false;
  int cur_job = -1;
  float2* const xa = X + T * kXP;
  float2* const xb = X + (4 * n2y) * kXP + k1lo;
  float2* const xc = X + (128 * k2x + k1y) * kXP + k1x;
  float2* const xw = X + (T >> 5) * (32 * kXP);
  const float2* const tr = xw + (ya & 7) * kTRow + ra;
  uint32_t phase = 0;   // parity of the next round of every tile's mbarrier
  // a wait that gives up sets `bad`; the TMEM load after it still reads this CTA's own
  // columns (values of no use), and the next CTA barrier (__syncthreads_or) abandons the launch
  bool bad = false;

  // one MMA round of this thread's tile: operands stored and fenced by every thread of the
  // tile, then issued by the elected thread; returns after the tile's products are in TMEM
  auto round = [&](auto inv) {
    tc::fence_async_smem();
    tc::fence_before();
    tc::tile_sync(tile);
    if (elected) {
      tc::fence_after();
      tc::issue_tile<decltype(inv)::value>(smA, smB, tmem, tile);
      tc::commit(mb);
    }
    bad |= !tc::wait_phase_warp(mb, phase);
    phase ^= 1;
    tc::fence_after();
  };

  for (int li = blockIdx.x; li < a.n_list; li += gridDim.x) {
    int jb = 0;
    while (jb + 1 < a.n_jobs && li >= a.start[jb + 1]) ++jb;
    const SliceJob& J = a.job[jb];
    __syncthreads();   // the previous item's reads of the table and of ptab are done
    if (jb != cur_job) {
      cur_job = jb;
      for (int e = T; e < kPTab; e += kThreads) {
        const int pa = e / kPRow, pb = e - pa * kPRow;
        const float2 v = cmul(J.ex[pa], J.ey[pb]);
        ptab[e] = pa * pa + pb * pb <= J.r2max ? make_float2(v.x * tc::kPropScale, v.y * tc::kPropScale)
                                               : make_float2(0.f, 0.f);
      }
      c_live = __any_sync(0xffffffffu, kxs * kxs <= J.r2max);
      __syncthreads();   // ptab complete
    }
    const int n_slices = J.n_slices;
    const int pitch = J.nx + kW;
    const size_t slice_elems = static_cast<size_t>(pitch) * (J.ny + kW);
    const int item = a.list[li];
    const int cfg = item / J.n_translates;
    const int ti = item - cfg * J.n_translates;
    const int ia = ti % J.lat_nax, ib = ti / J.lat_nax;
    int ox = (J.lat_ox + ia * J.lat_sx - kW / 2) % J.nx;
    if (ox < 0) ox += J.nx;
    int oy = (J.lat_oy + ib * J.lat_sy - kW / 2) % J.ny;
    if (oy < 0) oy += J.ny;
    const float2* const gsrc = J.t + cfg * J.t_slot + static_cast<size_t>(oy + 8 * (T >> 5)) * pitch + ox;

    stage_t_warp<EVEN>(xw, gsrc, pitch, lane);
    float2 v[32];
#pragma unroll
    for (int n1 = 0; n1 < 32; ++n1) {
      const float2 u = J.uW[ya * kW + 4 * n1 + ra];
      v[n1] = make_float2(u.x * J.tc_in, u.y * J.tc_in);
    }

    for (int s = 0; s < n_slices; ++s) {
      // transmission (Sec. 3.2), with the 2^-7 that the propagator leaves
      cp_async_wait_all();
      __syncwarp();
#pragma unroll
      for (int n1 = 0; n1 < 32; ++n1) {
        const float2 p = cmul(v[n1], tr[4 * n1]);
        v[n1] = make_float2(p.x * tc::kTransScale, p.y * tc::kTransScale);
      }
      // pass A forward: the tile's staged transmission rows are read before its operands
      // overwrite them
      tc::tile_sync(tile);
      tc::store_row(aHi, aLo, v, arow);
      round(std::false_type{});
      tc::load_row(t_row, v);
      // X1: this row's pass-A outputs, in the tile's own rows (its MMAs are complete)
      float4* const xa4 = reinterpret_cast<float4*>(xa);
#pragma unroll
      for (int k = 0; k < 32; k += 2) xa4[k / 2] = make_float4(v[k].x, v[k].y, v[k + 1].x, v[k + 1].y);
      if (__syncthreads_or(bad)) goto abort;
      float2 b0[16], b1[16];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          b0[q * 4 + r] = xb[(128 * q + r) * kXP];
          b1[q * 4 + r] = xb[(128 * q + r) * kXP + 16];
        }
      passB_fwd_tw<false, PRUNE>(b0, tB, twr[k1lo], twr[32 + k1lo]);
      passB_fwd_tw<true, PRUNE>(b1, tB, twr[16 + k1lo], twr[48 + k1lo]);
      static_for<0, 4>([&](auto qq) {
        constexpr int q = decltype(qq)::value;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          if constexpr (q != masked_k2x<false, PRUNE>()) xb[(128 * q + r) * kXP] = b0[r * 4 + q];
          if constexpr (q != masked_k2x<true, PRUNE>()) xb[(128 * q + r) * kXP + 16] = b1[r * 4 + q];
        }
      });
      __syncthreads();
      // pass C forward: every row of X2 is read before the operands overwrite the table
      float2 c[32];
      if (c_live) {
#pragma unroll
        for (int j = 0; j < 32; ++j) c[j] = xc[j * 4 * kXP];
      }
      __syncthreads();
      if (c_live) tc::store_row(aHi, aLo, c, arow);
      round(std::false_type{});
      if (c_live) {
        tc::load_row(t_row, c);
        // propagation (Sec. 3.2): exp(-i pi lambda eps |k|^2), bandlimit, 2^-7
#pragma unroll
        for (int j = 0; j < 32; ++j) c[j] = cmul(c[j], j < 16 ? pp[4 * j] : pm[-4 * j]);
        tc::store_row(aHi, aLo, c, arow);   // the tile's MMAs have read its operands
      }
      round(std::true_type{});
      if (c_live) tc::load_row(t_row, c);
      // X3 goes to every tile's rows: every tile's inverse products must be complete
#pragma unroll 1
      for (int u = 0; u < 4; ++u)
        if (u != tile) bad |= !tc::wait_phase_warp(tc::smem_u32(mbar + u), phase ^ 1);
      if (c_live) {
#pragma unroll
        for (int j = 0; j < 32; ++j) xc[j * 4 * kXP] = c[j];
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) xc[j * 4 * kXP] = make_float2(0.f, 0.f);
      }
      tc::fence_before();
      if (__syncthreads_or(bad)) goto abort;
      static_for<0, 4>([&](auto qq) {
        constexpr int q = decltype(qq)::value;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          if constexpr (q != masked_k2x<false, PRUNE>()) b0[r * 4 + q] = xb[(128 * q + r) * kXP];
          if constexpr (q != masked_k2x<true, PRUNE>()) b1[r * 4 + q] = xb[(128 * q + r) * kXP + 16];
        }
      });
      passB_inv_tw<false, PRUNE>(b0, tB, twr[k1lo], twr[32 + k1lo]);
      passB_inv_tw<true, PRUNE>(b1, tB, twr[16 + k1lo], twr[48 + k1lo]);
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          xb[(128 * q + r) * kXP] = b0[q * 4 + r];
          xb[(128 * q + r) * kXP + 16] = b1[q * 4 + r];
        }
      __syncthreads();
      {
        const float4* const xa4r = reinterpret_cast<const float4*>(xa);
#pragma unroll
        for (int k = 0; k < 32; k += 2) {
          const float4 p = xa4r[k / 2];
          v[k] = make_float2(p.x, p.y);
          v[k + 1] = make_float2(p.z, p.w);
        }
      }
      // pass A inverse: the tile's X4 rows (read only by the tile) are read before its
      // operands overwrite them
      tc::tile_sync(tile);
      tc::store_row(aHi, aLo, v, arow);
      round(std::true_type{});
      tc::load_row(t_row, v);
      // the tile's MMAs have read its rows: stage the next slice's transmission there
      __syncwarp();
      if (s + 1 < n_slices) stage_t_warp<EVEN>(xw, gsrc + (s + 1) * slice_elems, pitch, lane);
    }
    if (__syncthreads_or(bad)) goto abort;
    const int oi = a.out_index ? a.out_index[li] : ti;
    float2* ud = J.U + cfg * J.u_slot + static_cast<size_t>(oi) * (kW * kW) + ya * kW + ra;
#pragma unroll
    for (int n1 = 0; n1 < 32; ++n1) ud[4 * n1] = make_float2(v[n1].x * J.tc_out, v[n1].y * J.tc_out);
  }
  if (false) {
  abort:
    // a tensor-core wait gave up (the decision is CTA-uniform)
    bad = true;
  }
  cp_async_wait_all();
  if (bad) {
    if (T == 0) atomicOr(status, 1);
    // the tile's last MMA group may still be in flight: give it the same bounded wait
    // before freeing TMEM
    tc::wait_phase(mb, phase ^ 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tc::kTmemCols) : "memory");
}

// ------------------------------------------------------------------------------------------
// helpers of the W = 256 kernel's bulk copies (and the thread count of the W = 64 / 256 kernels)
// ------------------------------------------------------------------------------------------
namespace gen {

constexpr int kThreadsGen = 512;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

}  // namespace gen

// bulk-copy helpers of the W = 256 path (TMA engine, non-tensor form)
namespace gen {
__device__ __forceinline__ void expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
}  // namespace gen

// Self-test of the bounded waits: warps wait on phase 0 of an mbarrier that nothing completes,
// with the bounded warp wait of the tensor-core and W = 256 slice kernels (lane 0 suspended up
// to kSuspendLimit tries of kSuspendNs, then one try_wait per lane), in one warp (which = 0) or
// in the 16 warps of a W = 256 CTA (which = 1), and report the give-up in *status as those
// kernels do.
__global__ void k_selftest_wait(int* status) {
  __shared__ __align__(8) uint64_t mbar;
  const uint32_t mb = tc::smem_u32(&mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = tc::wait_phase_warp(mb, 0);
  if (!ok && (threadIdx.x & 31) == 0) atomicOr(status, 1);
}


// ------------------------------------------------------------------------------------------
// step a3 on W = 256 windows: each 256-point transform as two in-register 16-point passes
// ------------------------------------------------------------------------------------------
// With x = 16 n + q and k = k1 + 16 k2 (Cooley-Tukey, 256 = 16 x 16),
//   X[k1 + 16 k2] = sum_q W_16^(q k2) W_256^(q k1) sum_n W_16^(n k1) x[16 n + q].
// Pass 1: the thread of residue q takes x[16 n + q] (n < 16), takes the 16-point DFT over n,
// multiplies by W_256^(q k1) and puts the results back where it read them (entry 16 k1 + q).
// Pass 2: the thread of k1 takes entries 16 k1 + q (q < 16), takes the DFT over q and puts
// X[k1 + 16 k2] at entry 16 k1 + k2. The spectrum thus stays in digit-reversed order (entry
// 16 a + b holds frequency a + 16 b), where the propagator indexes it; the inverse runs the
// passes back with conjugate twiddles, each thread writing only entries it has just read.
//
// The wave lives in a per-CTA scratch in global memory (L2). Each slice is a column phase
// (forward over y, propagator, inverse over y) and a row phase (inverse over x, transmission
// of the next slice, forward over x), each over 8 panels of 32 columns or 32 rows (64 KiB),
// double-buffered in shared memory and moved by bulk copies completing on an mbarrier.
//   Column panel [256 y][34]: thread (c, g) = (lane, warp); pass 1 is residue q = g, pass 2
//   is k1 = g; CTA barriers between the passes. 32 lanes read 32 consecutive entries.
//   Row panel [32 r][256]: thread (r, j) = (2 warp + lane / 16, lane % 16), so that a row's
//   passes stay in one half-warp (__syncwarp between them). Scratch rows and row panels hold
//   entry p at the swizzled position swz(p) (low four bits XOR the high four): the pass-2
//   reads of entries 16 j + k2 and the pass-1 reads of 16 k1 + j then fall on 16 distinct
//   bank pairs, and a panel still moves as one contiguous bulk copy.
namespace w256 {
constexpr int kN = 256;
constexpr int kPanels = 8;
constexpr int kPC = 34;                  // column-panel row pitch (32 entries + 16-byte pad)
constexpr int kBuf = kN * kPC;           // float2 per panel buffer (a row panel takes 32 x 256)
// W_256^m = exp(-2 pi i m / 256), m < 256, built on the host in FP64 and rounded once
__constant__ float2 c_tw[kN];
__host__ __device__ constexpr int swz(int p) { return (p & ~15) | ((p & 15) ^ ((p >> 4) & 15)); }

// L2 policy of the scratch copies: keep the scratch resident (the exit waves stream past it)
__device__ __forceinline__ uint64_t policy_keep() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void load(void* smem_dst, const void* gsrc, uint32_t bytes, uint32_t mbar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          gen::smem_u32(smem_dst)),
      "l"(gsrc), "r"(bytes), "r"(mbar), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void store(void* gdst, const void* smem_src, uint32_t bytes, uint64_t pol) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(gdst),
               "r"(gen::smem_u32(smem_src)), "r"(bytes), "l"(pol)
               : "memory");
}

// column panel: forward over y, propagator and bandlimit, inverse over y (thread (c, g));
// eyt: the job's exp(-i pi lambda eps ky^2) in shared memory (read at warp-uniform ky)
__device__ __forceinline__ void column_panel(float2* buf, int p, const SliceJob& J, const float2* eyt, int c, int g) {
  float2 v[16];
#pragma unroll
  for (int n = 0; n < 16; ++n) v[n] = buf[(16 * n + g) * kPC + c];
  dft16<false>(v);
#pragma unroll
  for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], c_tw[g * k1]);
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) buf[(16 * k1 + g) * kPC + c] = v[k1];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = buf[(16 * g + q) * kPC + c];
  dft16<false>(v);
  // propagation (Sec. 3.2) at (kx, ky): the column at scratch position 32 p + c holds row entry
  // e = swz(32 p + c), frequency kx = e / 16 + 16 (e % 16); v[k2] has ky = g + 16 k2
  const int e = swz(32 * p + c);
  const int kxi = (e >> 4) + 16 * (e & 15);
  const int kxs = kxi < kN / 2 ? kxi : kxi - kN;
  const float2 ex = J.ex[kxi];
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) {
    const int kyi = g + 16 * k2;
    const int kys = kyi < kN / 2 ? kyi : kyi - kN;
    v[k2] = kxs * kxs + kys * kys <= J.r2max ? cmul(v[k2], cmul(ex, eyt[kyi])) : make_float2(0.f, 0.f);
  }
  dft16<true>(v);
#pragma unroll
  for (int q = 1; q < 16; ++q) v[q] = cmulc(v[q], c_tw[g * q]);
#pragma unroll
  for (int q = 0; q < 16; ++q) buf[(16 * g + q) * kPC + c] = v[q];
  __syncthreads();
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) v[k1] = buf[(16 * k1 + g) * kPC + c];
  dft16<true>(v);
#pragma unroll
  for (int n = 0; n < 16; ++n) buf[(16 * n + g) * kPC + c] = v[n];
}

// forward over x of one row (pass 1 from v[n] = x[16 n + j], then pass 2), into the panel row
__device__ __forceinline__ void row_forward(float2* row, float2 (&v)[16], int j, const float2 (&twj)[16]) {
  dft16<false>(v);
#pragma unroll
  for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], twj[k1]);
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) row[16 * k1 + (j ^ k1)] = v[k1];   // entry 16 k1 + j
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = row[16 * j + (q ^ j)];           // entry 16 j + q
  dft16<false>(v);
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) row[16 * j + (k2 ^ j)] = v[k2];      // entry 16 j + k2
}

// inverse over x of one row: v[n] = x[16 n + j] afterwards (the row's entries are consumed)
__device__ __forceinline__ void row_inverse(float2* row, float2 (&v)[16], int j, const float2 (&twj)[16]) {
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) v[k2] = row[16 * j + (k2 ^ j)];
  dft16<true>(v);
#pragma unroll
  for (int q = 1; q < 16; ++q) v[q] = cmulc(v[q], twj[q]);
#pragma unroll
  for (int q = 0; q < 16; ++q) row[16 * j + (q ^ j)] = v[q];
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) v[k1] = row[16 * k1 + (j ^ k1)];
  dft16<true>(v);
}
}  // namespace w256

// One translate per CTA at a time (persistent CTAs), complex64 exit waves, W = 256. scratch:
// 256 x 256 complex64 per CTA; status: set to 1 when a bulk-copy wait gives up.
//
// Column phase: the CTA moves panels of 32 columns (256 copies of 256 bytes, threads T < 256)
// through two buffers on two mbarriers; the next panel's load is issued before the current one
// is transformed (after the issuing thread's own previous store from that buffer has read it;
// the byte count may reach the mbarrier before or after the copies do). Row phase: each warp
// moves its own two rows of each panel (one 4 KiB copy in, one out, by lane 0) through its
// two row slots on its own two mbarriers, so the row phase has no CTA barrier. Every wait is
// one polling lane per warp (bounded, suspended tries) and then one try_wait per lane. Scratch
// copies carry an evict-last L2 policy; the exit wave is written with streaming stores.
__global__ void __launch_bounds__(gen::kThreadsGen, 1) k_slice_256(const SliceLaunch a, float2* scratch, int* status) {
  using namespace w256;
  extern __shared__ __align__(16) unsigned char smg[];
  float2* const S = reinterpret_cast<float2*>(smg);
  float2* const eyt = S + 2 * kBuf;                                  // the job's ey, kN entries
  // mbarriers: [0, 2) column buffers; 2 + 2 w + b: row slot b of warp w
  uint64_t* const mbar = reinterpret_cast<uint64_t*>(eyt + kN);
  const int T = threadIdx.x, warp = T >> 5, lane = T & 31;
  const int rr = 2 * warp + (lane >> 4), jj = lane & 15;   // row-phase thread (r, j)
  // W_256^(j m): this thread's row-phase twiddles, read once (a constant read whose address
  // differs across a warp is serialized)
  float2 twj[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) twj[m] = c_tw[jj * m];
  float2* const G = scratch + static_cast<size_t>(blockIdx.x) * kN * kN;
  const uint64_t keep = policy_keep();
  if (T < 2 + 2 * (gen::kThreadsGen / 32)) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(gen::smem_u32(mbar + T)) : "memory");
    if (T == 0) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const uint32_t mrow = gen::smem_u32(mbar + 2 + 2 * warp);        // this warp's row mbarriers (+ 8 b)
  uint32_t phc = 0u, phr = 0u;                                      // completed-phase parity per buffer
  bool bad = false;
  int cur_job = -1;
  constexpr uint32_t kRowBytes = 2 * kN * 8;                         // a warp's two rows

  for (int li = blockIdx.x; li < a.n_list; li += gridDim.x) {
    int jb = 0;
    while (jb + 1 < a.n_jobs && li >= a.start[jb + 1]) ++jb;
    const SliceJob& J = a.job[jb];
    const int n_slices = J.n_slices;
    const int pitch = J.nx + kW;                          // padded transmission row
    const size_t slice_elems = static_cast<size_t>(pitch) * (J.ny + kW);
    const int item = a.list[li];
    const int cfg = item / J.n_translates;
    const int ti = item - cfg * J.n_translates;
    const int ia = ti % J.lat_nax, ib = ti / J.lat_nax;
    int ox = (J.lat_ox + ia * J.lat_sx - kN / 2) % J.nx;
    if (ox < 0) ox += J.nx;
    int oy = (J.lat_oy + ib * J.lat_sy - kN / 2) % J.ny;
    if (oy < 0) oy += J.ny;
    const float2* const tbase = J.t + cfg * J.t_slot;
    // transmission of slice s at window pixel (y, x): the periodic cell, indices wrapped (the
    // halo of the stored array is narrower than this window)
    auto tval = [&](int s, int y, int x) -> float2 {
      int gy = oy + y, gx = ox + x;
      if (gy >= J.ny) gy -= J.ny;
      if (gx >= J.nx) gx -= J.nx;
      return tbase[s * slice_elems + static_cast<size_t>(gy) * pitch + gx];
    };
    const int oi = a.out_index ? a.out_index[li] : ti;
    float2* const ud = J.U + cfg * J.u_slot + static_cast<size_t>(oi) * (kN * kN);
    __syncthreads();   // the previous item's use of the buffers and of eyt is over
    if (n_slices == 0) {
      for (int e = T; e < kN * kN; e += gen::kThreadsGen) ud[e] = J.uW[e];
      continue;
    }
    if (jb != cur_job) {
      cur_job = jb;
      for (int e = T; e < kN; e += gen::kThreadsGen) eyt[e] = J.ey[e];   // read after the barriers below
    }
    // rows of the scratch: input wave times the transmission of slice 0, forward over x (each
    // warp its own two rows per panel, alternating row slots)
    for (int p = 0; p < kPanels; ++p) {
      float2* const slot = S + (p & 1) * kBuf + 2 * warp * kN;
      if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");   // slot's store of p - 2
      __syncwarp();
      const int y = 32 * p + rr;
      float2 v[16];
#pragma unroll
      for (int n = 0; n < 16; ++n) v[n] = cmul(J.uW[y * kN + 16 * n + jj], tval(0, y, 16 * n + jj));
      row_forward(S + (p & 1) * kBuf + rr * kN, v, jj, twj);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        store(G + static_cast<size_t>(32 * p + 2 * warp) * kN, slot, kRowBytes, keep);
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    for (int s = 0; s < n_slices && !bad; ++s) {
      // ---- column phase ----
      auto issue_col = [&](int pn) {
        const int bn = pn & 1;
        const uint32_t mb = gen::smem_u32(mbar + bn);
        if (T == 0) gen::expect_tx(mb, 32u * kN * 8u);
        if (T < kN) load(S + bn * kBuf + T * kPC, G + static_cast<size_t>(T) * kN + pn * 32, 32 * 8, mb, keep);
      };
      issue_col(0);
      for (int p = 0; p < kPanels; ++p) {
        const int b = p & 1;
        float2* const buf = S + b * kBuf;
        if (p + 1 < kPanels) {
          // this thread's store of panel p - 1 has read its part of the other buffer
          if (T < kN) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
          issue_col(p + 1);
        }
        bad |= !tc::wait_phase_warp(gen::smem_u32(mbar + b), (phc >> b) & 1u);
        phc ^= 1u << b;
        column_panel(buf, p, J, eyt, lane, warp);
        // the threads' writes are made visible to the bulk copies, then the panel goes back
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (T < kN) {
          store(G + static_cast<size_t>(T) * kN + p * 32, buf + T * kPC, 32 * 8, keep);
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
      }
      // every store of the phase is complete before the row phase reads the scratch
      if (T < kN) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
      asm volatile("fence.proxy.async.global;" ::: "memory");
      __syncthreads();
      // ---- row phase: each warp its own two rows of every panel ----
      const bool last = s + 1 == n_slices;   // rows go to the exit wave, not back
      auto issue_row = [&](int pn) {
        if (lane == 0) {
          const uint32_t mb = mrow + 8 * (pn & 1);
          gen::expect_tx(mb, kRowBytes);
          load(S + (pn & 1) * kBuf + 2 * warp * kN, G + static_cast<size_t>(32 * pn + 2 * warp) * kN, kRowBytes, mb, keep);
        }
      };
      issue_row(0);
      for (int p = 0; p < kPanels; ++p) {
        const int b = p & 1;
        if (p + 1 < kPanels) {
          if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");   // slot's store of p - 1
          issue_row(p + 1);
        }
        bad |= !tc::wait_phase_warp(mrow + 8 * b, (phr >> b) & 1u);
        phr ^= 1u << b;
        float2* const row = S + b * kBuf + rr * kN;
        const int y = 32 * p + rr;
        float2 v[16];
        row_inverse(row, v, jj, twj);
        if (last) {
#pragma unroll
          for (int n = 0; n < 16; ++n) __stcs(ud + y * kN + 16 * n + jj, v[n]);
          __syncwarp();   // every lane has read the slot before lane 0 loads the next panel into it
        } else {
#pragma unroll
          for (int n = 0; n < 16; ++n) v[n] = cmul(v[n], tval(s + 1, y, 16 * n + jj));
          row_forward(row, v, jj, twj);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) {
            store(G + static_cast<size_t>(32 * p + 2 * warp) * kN, S + b * kBuf + 2 * warp * kN, kRowBytes, keep);
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          }
        }
      }
      if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
      asm volatile("fence.proxy.async.global;" ::: "memory");
      bad = __syncthreads_or(bad);
    }
    if (__syncthreads_or(bad)) break;
  }
  if (bad && T == 0) atomicOr(status, 1);
}

// ------------------------------------------------------------------------------------------
// step a3 on W = 64 windows: each 64-point transform as two in-register 8-point passes
// ------------------------------------------------------------------------------------------
// 64 = 8 x 8 as for W = 256: with x = 8 n + q and k = k1 + 8 k2, pass 1 takes the 8-point DFT
// over n for residue q and multiplies by W_64^(q k1), pass 2 the DFT over q for k1; the
// spectrum stays in digit-reversed order (entry 8 a + b holds frequency a + 8 b). The wave
// (32 KiB) stays in shared memory in two buffers of opposite orientation, A[y][x] and
// B[x][y] (rows of 65 entries). A phase reads one buffer with thread (c, g): c the position
// along the other axis (the 32 lanes of a warp on consecutive positions), g = warp / 2 the
// residue (pass 1) or k1 (pass 2); its passes work in place between CTA barriers, and it
// writes its result transposed into the other buffer, so that the row phase runs the column
// phase's code on B. Column phase: forward over y, propagator, inverse over y (A -> B). Row
// phase: inverse over x, the next slice's transmission, forward over x (B -> A). The next
// slice's transmission is staged into a third buffer by 8-byte cp.async while the column
// phase runs. About 100 KB of shared memory: two CTAs per SM.
namespace w64 {
constexpr int kN = 64;
constexpr int kP = 65;                   // buffer row pitch (64-bit accesses of 16 lanes at stride 65 or 1: 32 banks)
constexpr int kBufE = kN * kP;           // float2 per buffer
// W_64^m = exp(-2 pi i m / 64), m < 64, built on the host in FP64 and rounded once
__constant__ float2 c_tw[kN];

// in-register 8-point DFT, natural order in and out: the first three stages of dft32
template <bool INV>
__device__ __forceinline__ void dft8(float2 (&v)[8]) {
  float2 t[8];
  static_for<0, 8>([&](auto k) {
    constexpr int K = decltype(k)::value;
    t[K] = v[((K & 1) << 2) | (K & 2) | ((K & 4) >> 2)];
  });
  static_for<0, 3>([&](auto st) {
    constexpr int H = 1 << decltype(st)::value;
    static_for<0, 4 / H>([&](auto blk) {
      static_for<0, H>([&](auto j) {
        constexpr int I = decltype(blk)::value * 2 * H + decltype(j)::value;
        constexpr int M = decltype(j)::value * (16 / H);
        bfly<INV, I, H, M>(t);
      });
    });
  });
  static_for<0, 8>([&](auto k) {
    constexpr int K = decltype(k)::value;
    v[K] = t[K];
  });
}

// forward over one axis for thread (c, g) of buffer X: pass 1 from v[n] = x[8 n + g] (already
// in registers), pass 2; X[entry][c] is the in-place scratch; v[k2] = X[g + 8 k2] after it
__device__ __forceinline__ void forward(float2* X, float2 (&v)[8], int c, int g) {
  dft8<false>(v);
#pragma unroll
  for (int k1 = 1; k1 < 8; ++k1) v[k1] = cmul(v[k1], c_tw[g * k1]);
#pragma unroll
  for (int k1 = 0; k1 < 8; ++k1) X[(8 * k1 + g) * kP + c] = v[k1];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = X[(8 * g + q) * kP + c];
  dft8<false>(v);
}
// inverse over one axis for thread (c, g), from v[k2] = X[g + 8 k2] (in registers); v[n] =
// x[8 n + g] after it
__device__ __forceinline__ void inverse(float2* X, float2 (&v)[8], int c, int g) {
  dft8<true>(v);
#pragma unroll
  for (int q = 1; q < 8; ++q) v[q] = cmulc(v[q], c_tw[g * q]);
#pragma unroll
  for (int q = 0; q < 8; ++q) X[(8 * g + q) * kP + c] = v[q];
  __syncthreads();
#pragma unroll
  for (int k1 = 0; k1 < 8; ++k1) v[k1] = X[(8 * k1 + g) * kP + c];
  dft8<true>(v);
}
}  // namespace w64

// One translate per CTA at a time (persistent CTAs, two per SM), complex64 exit waves, W = 64.
__global__ void __launch_bounds__(512, 2) k_slice_64(const SliceLaunch a) {
  using namespace w64;
  extern __shared__ __align__(16) float2 s64[];
  float2* const A = s64;                 // A[y][x entry]
  float2* const B = A + kBufE;           // B[x][y]
  float2* const Tb = B + kBufE;          // staged transmission [y][x]
  float2* const eyt = Tb + kBufE;        // the job's ey
  const int T = threadIdx.x, lane = T & 31, warp = T >> 5;
  const int c = lane + 32 * (warp & 1), g = warp >> 1;
  int cur_job = -1;
  for (int li = blockIdx.x; li < a.n_list; li += gridDim.x) {
    int jb = 0;
    while (jb + 1 < a.n_jobs && li >= a.start[jb + 1]) ++jb;
    const SliceJob& J = a.job[jb];
    const int n_slices = J.n_slices;
    const int pitch = J.nx + kW;                          // padded transmission row
    const size_t slice_elems = static_cast<size_t>(pitch) * (J.ny + kW);
    const int item = a.list[li];
    const int cfg = item / J.n_translates;
    const int ti = item - cfg * J.n_translates;
    const int ia = ti % J.lat_nax, ib = ti / J.lat_nax;
    int ox = (J.lat_ox + ia * J.lat_sx - kN / 2) % J.nx;
    if (ox < 0) ox += J.nx;
    int oy = (J.lat_oy + ib * J.lat_sy - kN / 2) % J.ny;
    if (oy < 0) oy += J.ny;
    // the halo of kW >= 64 pixels keeps every window inside the padded array
    const float2* const tw0 = J.t + cfg * J.t_slot + static_cast<size_t>(oy) * pitch + ox;
    const int oi = a.out_index ? a.out_index[li] : ti;
    float2* const ud = J.U + cfg * J.u_slot + static_cast<size_t>(oi) * (kN * kN);
    __syncthreads();   // the previous item's use of the buffers is over
    if (n_slices == 0) {
      for (int e = T; e < kN * kN; e += 512) ud[e] = J.uW[e];
      continue;
    }
    if (jb != cur_job) {
      cur_job = jb;
      if (T < kN) eyt[T] = J.ey[T];
    }
    // slice s's transmission window into Tb (coalesced rows, asynchronous)
    auto stage = [&](int s) {
      const float2* const src = tw0 + static_cast<size_t>(s) * slice_elems;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int e = T + 512 * i, y = e >> 6, x = e & 63;
        cp_async8(Tb + y * kP + x, src + static_cast<size_t>(y) * pitch + x);
      }
      cp_async_commit();
    };
    stage(0);
    cp_async_wait_all();
    __syncthreads();
    {
      // rows y = c: the input wave times the transmission of slice 0, forward over x into A
      float2 v[8];
#pragma unroll
      for (int n = 0; n < 8; ++n) v[n] = cmul(J.uW[c * kN + 8 * n + g], Tb[c * kP + 8 * n + g]);
      forward(B, v, c, g);
#pragma unroll
      for (int k2 = 0; k2 < 8; ++k2) A[c * kP + 8 * g + k2] = v[k2];
    }
    // propagator of this thread's column phase: the column at x entry c holds kx = c / 8 + 8 (c % 8)
    const int kxi = (c >> 3) + 8 * (c & 7);
    const int kxs = kxi < kN / 2 ? kxi : kxi - kN;
    const float2 ex = J.ex[kxi];
    __syncthreads();
    for (int s = 0; s < n_slices; ++s) {
      if (s + 1 < n_slices) stage(s + 1);   // Tb's last reads (slice s's transmission) are done
      // column phase: x entry c, forward over y, propagation (Sec. 3.2), inverse over y, into B
      {
        float2 v[8];
#pragma unroll
        for (int n = 0; n < 8; ++n) v[n] = A[(8 * n + g) * kP + c];
        forward(A, v, c, g);
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) {
          const int kyi = g + 8 * k2;
          const int kys = kyi < kN / 2 ? kyi : kyi - kN;
          v[k2] = kxs * kxs + kys * kys <= J.r2max ? cmul(v[k2], cmul(ex, eyt[kyi])) : make_float2(0.f, 0.f);
        }
        inverse(A, v, c, g);
#pragma unroll
        for (int n = 0; n < 8; ++n) B[c * kP + 8 * n + g] = v[n];
      }
      cp_async_wait_all();
      __syncthreads();
      // row phase: row y = c, inverse over x, the next slice's transmission, forward over x, into A
      {
        float2 v[8];
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) v[k2] = B[(8 * g + k2) * kP + c];
        inverse(B, v, c, g);
        if (s + 1 < n_slices) {
#pragma unroll
          for (int n = 0; n < 8; ++n) v[n] = cmul(v[n], Tb[c * kP + 8 * n + g]);
          forward(B, v, c, g);
#pragma unroll
          for (int k2 = 0; k2 < 8; ++k2) A[c * kP + 8 * g + k2] = v[k2];
        } else {
#pragma unroll
          for (int n = 0; n < 8; ++n) A[c * kP + 8 * n + g] = v[n];   // natural x: the exit wave
        }
      }
      __syncthreads();
    }
    for (int e = T; e < kN * kN; e += 512) ud[e] = A[(e >> 6) * kP + (e & 63)];
  }
}

// ------------------------------------------------------------------------------------------
// step a3, real-space variant: the propagation step as a convolution with the K1 x K2
// kernel q (Sec. 3.2, complexity paragraph). One CTA per translate, the wave in shared
// memory; thread (lane, warp) accumulates the 32 outputs x = lane + 32 m (m < 4), y =
// 8 warp + j (j < 8) in registers: out(x, y) = sum over offsets (oy, ox) of q(oy, ox) psi(y -
// oy, x - ox), periodic on the window. MB columns share one register segment of K1 inputs
// (up to 13 at a time: K1 from 15 to 25 takes the segment in two pieces).
// ------------------------------------------------------------------------------------------
// One input row u of the convolution for the kernels with K2 fixed at compile time: its
// segment of K1 inputs per output column (in pieces of KC), applied to every output row j
// it feeds (kernel row dyi = j - u + h). The runtime-K2 kernels keep the same steps written
// inline in their input-row loop (measured 2 % faster there at K = 13 and 25).
template <int K1, int MB, int KC>
__device__ __forceinline__ void rs_row_step(float2 (&acc)[8][4], const float2* psi, const float2* q, int wy,
                                            int lane, int mb, int u, int h, int K2) {
  const float2* row = psi + ((8 * wy + u) & (kW - 1)) * kW;
#pragma unroll
  for (int c0 = 0; c0 < K1; c0 += KC) {
    float2 seg[MB][KC];
#pragma unroll
    for (int mm = 0; mm < MB; ++mm)
#pragma unroll
      for (int d = 0; d < KC; ++d)
        if (c0 + d < K1) seg[mm][d] = row[(lane + 32 * (mb + mm) - (c0 + d - K1 / 2)) & (kW - 1)];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int dyi = j - u + h;
      if (dyi < 0 || dyi >= K2) continue;
      const float2* qr = q + dyi * K1 + c0;
#pragma unroll
      for (int d = 0; d < KC; ++d) {
        if (c0 + d >= K1) continue;
        const float2 qv = qr[d];
#pragma unroll
        for (int mm = 0; mm < MB; ++mm) acc[j][mb + mm] = cfma(acc[j][mb + mm], qv, seg[mm][d]);
      }
    }
  }
}

// K2F > 0 fixes K2 at compile time (the small square kernels): the input-row loop then
// unrolls, its row-range tests fold away and q is read at constant offsets. These kernels
// also apply each slice's transmission as the previous convolution's outputs are written
// (FUSE), instead of in a pass of its own over the wave in shared memory; the products
// and their order are the same.
template <int K1, int MB, int K2F = 0>
__global__ void __launch_bounds__(kThreads, 1) k_slice_rs(const SliceLaunch a, const float2* qg, const int K2arg) {
  constexpr bool FUSE = K2F > 0;
  const int K2 = K2F > 0 ? K2F : K2arg;
  extern __shared__ __align__(16) float2 sm[];
  float2* psi = sm;                 // [W][W]
  float2* q = sm + kW * kW;         // [K2][K1]
  const int T = threadIdx.x, lane = T & 31, wy = T >> 5;
  for (int i = T; i < K1 * K2; i += kThreads) q[i] = qg[i];
  for (int li = blockIdx.x; li < a.n_list; li += gridDim.x) {
    int jb = 0;
    while (jb + 1 < a.n_jobs && li >= a.start[jb + 1]) ++jb;
    const SliceJob& J = a.job[jb];
    const int item = a.list[li];
    const int cfg = item / J.n_translates;
    const int ti = item - cfg * J.n_translates;
    const int ia = ti % J.lat_nax, ib = ti / J.lat_nax;
    int ox = (J.lat_ox + ia * J.lat_sx - kW / 2) % J.nx;
    if (ox < 0) ox += J.nx;
    int oy = (J.lat_oy + ib * J.lat_sy - kW / 2) % J.ny;
    if (oy < 0) oy += J.ny;
    const int pitch = J.nx + kW;
    const size_t slice_elems = static_cast<size_t>(pitch) * (J.ny + kW);
    const float2* tb = J.t + cfg * J.t_slot + static_cast<size_t>(oy) * pitch + ox;
    __syncthreads();   // the previous item's reads of psi are done
    if (FUSE && J.n_slices > 0) {
      // the first slice's transmission applied as the input wave is loaded
      for (int p = T; p < kW * kW; p += kThreads)
        psi[p] = cmul(J.uW[p], tb[static_cast<size_t>(p >> 7) * pitch + (p & (kW - 1))]);
    } else {
      for (int p = T; p < kW * kW; p += kThreads) psi[p] = J.uW[p];
    }
    for (int s = 0; s < J.n_slices; ++s) {
      if constexpr (!FUSE) {
        // transmission (Sec. 3.2): psi <- t_s psi
        __syncthreads();
        const float2* ts = tb + s * slice_elems;
        // all 32 loads of this thread's transmission values first (row (T >> 7) + 4 i,
        // column T & 127), then the products
        float2 tv[kW * kW / kThreads];
#pragma unroll
        for (int i = 0; i < kW * kW / kThreads; ++i)
          tv[i] = ts[static_cast<size_t>((T >> 7) + 4 * i) * pitch + (T & 127)];
#pragma unroll
        for (int i = 0; i < kW * kW / kThreads; ++i) psi[T + kThreads * i] = cmul(psi[T + kThreads * i], tv[i]);
      }
      __syncthreads();
      // propagation: periodic convolution with q
      float2 acc[8][4];
#pragma unroll
      for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int m = 0; m < 4; ++m) acc[j][m] = make_float2(0.f, 0.f);
      // input rows in the outer loop: row 8 wy + u feeds output rows j with dyi = j - u + h
      // in [0, K2), so each input segment is read once for all of them (8 + K2 - 1 rows
      // instead of 8 K2)
      // kernels wider than 13 columns take their row segment in pieces of at most 13 (the
      // register footprint of the 13-column kernel); narrower ones in one piece
      const int h = K2 / 2;
      constexpr int KC = K1 < 13 ? K1 : 13;
#pragma unroll
      for (int mb = 0; mb < 4; mb += MB) {
        if constexpr (K2F > 0) {
#pragma unroll
          for (int u = K2F / 2 - (K2F - 1); u <= 7 + K2F / 2; ++u)
            rs_row_step<K1, MB, KC>(acc, psi, q, wy, lane, mb, u, h, K2);
        } else {
#pragma unroll 1
          for (int u = h - (K2 - 1); u <= 7 + h; ++u) {
            const float2* row = psi + ((8 * wy + u) & (kW - 1)) * kW;
#pragma unroll
            for (int c0 = 0; c0 < K1; c0 += KC) {
              float2 seg[MB][KC];
#pragma unroll
              for (int mm = 0; mm < MB; ++mm)
#pragma unroll
                for (int d = 0; d < KC; ++d)
                  if (c0 + d < K1) seg[mm][d] = row[(lane + 32 * (mb + mm) - (c0 + d - K1 / 2)) & (kW - 1)];
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int dyi = j - u + h;
                if (dyi < 0 || dyi >= K2) continue;
                const float2* qr = q + dyi * K1 + c0;
#pragma unroll
                for (int d = 0; d < KC; ++d) {
                  if (c0 + d >= K1) continue;
                  const float2 qv = qr[d];
#pragma unroll
                  for (int mm = 0; mm < MB; ++mm) acc[j][mb + mm] = cfma(acc[j][mb + mm], qv, seg[mm][d]);
                }
              }
            }
          }
        }
      }
      if constexpr (FUSE) {
        // the outputs times the next slice's transmission at the same pixels (rows 8 wy + j,
        // columns lane + 32 m), in two halves of 16 loads; the first half is in flight
        // while the CTA waits for every read of psi to finish
        const bool more = s + 1 < J.n_slices;
        const float2* tn = more ? tb + (s + 1) * slice_elems + static_cast<size_t>(8 * wy) * pitch + lane : nullptr;
        float2 tv[4][4];
        if (more) {
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int m = 0; m < 4; ++m) tv[j][m] = tn[static_cast<size_t>(j) * pitch + 32 * m];
        }
        __syncthreads();
        if (more) {
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int m = 0; m < 4; ++m) psi[(8 * wy + j) * kW + lane + 32 * m] = cmul(acc[j][m], tv[j][m]);
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int m = 0; m < 4; ++m) tv[j][m] = tn[static_cast<size_t>(4 + j) * pitch + 32 * m];
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int m = 0; m < 4; ++m) psi[(8 * wy + 4 + j) * kW + lane + 32 * m] = cmul(acc[4 + j][m], tv[j][m]);
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int m = 0; m < 4; ++m) psi[(8 * wy + j) * kW + lane + 32 * m] = acc[j][m];
        }
      } else {
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
          for (int m = 0; m < 4; ++m) psi[(8 * wy + j) * kW + lane + 32 * m] = acc[j][m];
      }
    }
    __syncthreads();
    const int oi = a.out_index ? a.out_index[li] : ti;
    float2* ud = J.U + cfg * J.u_slot + static_cast<size_t>(oi) * (kW * kW);
    for (int p = T; p < kW * kW; p += kThreads) ud[p] = psi[p];
  }
}

// ------------------------------------------------------------------------------------------
// steps a4-a6: synthesis and detector reading
// ------------------------------------------------------------------------------------------
constexpr int kSynthSmemFloat2 = kX1 + kTwA + 128 + (kThreads / 32) * kMaxDet;

// Probe of visit index q: the region is walked in vertical strips of sw columns (the
// last strip narrower), row by row within a strip. The CTAs in flight then read the
// exit waves of a compact patch of translates, which stays in L2 while the strip moves
// down; a raster walk over whole rows needs about seven 128-translate rows at once.
__device__ __forceinline__ int probe_of(int q, int npx, int npy, int sw) {
  const int per = npy * sw;
  const int s = q / per;
  const int x0 = s * sw;
  const int w = min(sw, npx - x0);
  const int r = q - s * per;
  return (r / w) * npx + x0 + (r - (r / w) * w);
}

// HALF reads the FP16 store and folds each wave's factor into its coefficient. MODE
// selects the readout (ReadMode): 2D annuli, labelled pixel sets (3D STEM rings) or the
// diffraction pattern on a centred crop (4D STEM).
// WS: the exit-wave window at compile time (kW), or 0 to take it from a.W (windows of other
// sizes, non-periodic placement only)
template <bool HALF, int MODE, bool CYCLIC, int WS = kW>
__global__ void __launch_bounds__(kThreads, 1) k_synth_detect(const SynthArgs a) {
  extern __shared__ __align__(16) float2 sm[];
  float2* R0 = sm;
  float2* twA = sm + kX1;
  float2* twB = twA + kTwA;
  float* red = reinterpret_cast<float*>(twB + 128);   // [16 warps][kMaxDet]

  const int T = threadIdx.x;
  load_twiddles(twA, twB, T);
  const int ra = T & 3;
  const int k1lo = T & 15, n2y = T >> 4;
  const int kx = c_column(T), k1y = T >> 7, k1x = kx & 31, k2x = kx >> 5;
  const float2* tA = twA + ra * 34;
  const float2* tB = twB + n2y * 4;
  float4* const x1w = reinterpret_cast<float4*>(R0 + T * 34);
  float2* const x1r = R0 + (4 * n2y) * 34 + k1lo;
  float2* const x2b = R0 + n2y * 32 + k1lo;
  float2* const x2c = R0 + (k1y * 4 + k2x) * 1024 + k1x;
  uint32_t dbits[kMaxDet];
  uint32_t any_bits = 0u;
  const int kxs = kx < 64 ? kx : kx - 128;
  if constexpr (MODE == kReadAnnuli) {
#pragma unroll
    for (int d = 0; d < kMaxDet; ++d) {
      dbits[d] = d < a.n_det ? a.det_bits[d * kThreads + kx + 128 * k1y] : 0u;
      any_bits |= dbits[d];
    }
  } else {
    // labels and the pattern cover in-band pixels only
    any_bits = kxs * kxs <= a.band_r2 ? 1u : 0u;
  }
  // a warp whose columns meet no detector skips pass C
  const bool c_live = __any_sync(0xffffffffu, any_bits != 0u);
  __syncthreads();

  // exit-wave window W (the store's row length); the probe window D is kW. The periodic
  // placement (CYCLIC) has W = D = kW.
  static_assert(!CYCLIC || WS == kW, "periodic placement has W = D");
  const int Wu = WS > 0 ? WS : a.W;
  const int n_walk = a.probe_list ? a.n_list : a.n_probes;
  const int n_items = n_walk * a.n_cfg;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int cfg = item / n_walk;
    const int q = item - cfg * n_walk;
    // p: the probe's region index (accumulator); tq: its row of the probe tables
    const int p = a.probe_list ? a.probe_list[q] : probe_of(q, a.npx, a.npy, a.strip);
    const int tq = a.probe_list ? q : p;
    const float2* const Uc = a.U ? a.U + cfg * a.u_slot : nullptr;
    const void* const Uhc = a.Uh ? static_cast<const void*>(static_cast<const __half2*>(a.Uh) + cfg * a.u_slot) : nullptr;
    const float* const Usc = a.Uscale ? a.Uscale + static_cast<size_t>(cfg) * a.n_translates : nullptr;
    // Accumulation layout: lane l of warp w holds, for window rows y = 8 w + yl (yl < 8),
    // columns x = 64 k + 2 l + e (k, e < 2) at acc[yl * 4 + k * 2 + e], so that one load
    // instruction of a warp reads 512 contiguous bytes of a translate row (256 from the
    // FP16 store). Pass A's layout (thread (y, r): x = 4 n1 + r) is reached afterwards
    // through the warp's own rows of the X1 table.
    float2 acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = make_float2(0.f, 0.f);
    const int32_t* tp = a.tidx + static_cast<size_t>(tq) * a.L;
    const float2* ap = a.alpha + static_cast<size_t>(tq) * a.L;
    const int2* sp = a.shift + static_cast<size_t>(tq) * a.L;
    const int warp_id = T >> 5, lane_id = T & 31;
    for (int j = 0; j < a.L; ++j) {
      float2 al = ap[j];
      const int2 sh = sp[j];
      const int ti = tp[j];
      if constexpr (HALF) {
        const float f = Usc[ti];
        al.x *= f;
        al.y *= f;
      }
      const float4 al4 = make_float4(al.x, al.x, -al.y, al.y);   // cfma2's form of the coefficient
      const bool pair = (sh.x & 1) == 0;   // column pairs stay aligned and unbroken
      if (pair) {
        // all 16 loads of this translate first (pairs outside a non-periodic window read
        // as zero), then the 32 complex FMAs; the FP16 store is kept packed until then
        using Raw = typename std::conditional<HALF, uint2, float4>::type;
        Raw buf[16];
        if constexpr (!CYCLIC) {
          // one pointer per translate, the 16 loads at fixed offsets (rows yl, halves kk);
          // rows and columns outside the window are predicated off
          // element (y0 + yl, x0 + 64 kk) of translate ti is at signed offset base + yl W +
          // 64 kk; only offsets of rows and columns inside the window are dereferenced
          const int y0 = 8 * warp_id - sh.y, x0 = 2 * lane_id - sh.x;
          const long long base = static_cast<long long>(ti) * (Wu * Wu) + y0 * Wu + x0;
          const bool okx0 = static_cast<unsigned>(x0) < static_cast<unsigned>(Wu);
          const bool okx1 = static_cast<unsigned>(x0 + 64) < static_cast<unsigned>(Wu);
#pragma unroll
          for (int yl = 0; yl < 8; ++yl) {
            const bool oky = static_cast<unsigned>(y0 + yl) < static_cast<unsigned>(Wu);
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
              Raw r{};
              if (oky && (kk ? okx1 : okx0)) {
                const long long e = base + (yl * Wu + 64 * kk);
                if constexpr (HALF)
                  r = *reinterpret_cast<const uint2*>(static_cast<const __half2*>(Uhc) + e);
                else
                  r = *reinterpret_cast<const float4*>(Uc + e);
              }
              buf[yl * 2 + kk] = r;
            }
          }
        } else {
#pragma unroll
        for (int yl = 0; yl < 8; ++yl) {
          int yy = 8 * warp_id + yl - sh.y;
          bool ok = true;
          if constexpr (CYCLIC)
            yy &= (kW - 1);
          else
            ok = yy >= 0 && yy < Wu;
          const size_t off = static_cast<size_t>(ti) * (Wu * Wu) + yy * Wu;
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            int xp = 64 * kk + 2 * lane_id - sh.x;
            bool okx = ok;
            if constexpr (CYCLIC)
              xp &= (kW - 1);
            else
              okx = okx && xp >= 0 && xp < Wu;
            Raw r{};
            if (okx) {
              if constexpr (HALF)
                r = *reinterpret_cast<const uint2*>(static_cast<const __half2*>(Uhc) + off + xp);
              else
                r = *reinterpret_cast<const float4*>(Uc + off + xp);
            }
            buf[yl * 2 + kk] = r;
          }
        }
        }
#pragma unroll
        for (int b = 0; b < 16; ++b) {
          float2 f0, f1;
          if constexpr (HALF) {
            f0 = __half22float2(*reinterpret_cast<const __half2*>(&buf[b].x));
            f1 = __half22float2(*reinterpret_cast<const __half2*>(&buf[b].y));
          } else {
            f0 = make_float2(buf[b].x, buf[b].y);
            f1 = make_float2(buf[b].z, buf[b].w);
          }
          acc[2 * b] = cfma2(acc[2 * b], al4, f0);
          acc[2 * b + 1] = cfma2(acc[2 * b + 1], al4, f1);
        }
      } else {
#pragma unroll
        for (int yl = 0; yl < 8; ++yl) {
          int yy = 8 * warp_id + yl - sh.y;
          if constexpr (CYCLIC) {
            yy &= (kW - 1);
          } else if (yy < 0 || yy >= Wu) {
            continue;
          }
          const size_t off = static_cast<size_t>(ti) * (Wu * Wu) + yy * Wu;
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            int xe = 64 * (m >> 1) + 2 * lane_id + (m & 1) - sh.x;
            if constexpr (CYCLIC) {
              xe &= (kW - 1);
            } else if (xe < 0 || xe >= Wu) {
              continue;
            }
            if constexpr (HALF)
              acc[yl * 4 + m] = cfma(acc[yl * 4 + m], al, __half22float2(static_cast<const __half2*>(Uhc)[off + xe]));
            else
              acc[yl * 4 + m] = cfma(acc[yl * 4 + m], al, Uc[off + xe]);
          }
        }
      }
    }
    __syncthreads();   // previous probe's C reads of the table are done
    // warp-private transpose through the warp's X1 rows (1088 entries): element (yl, x) at
    // yl * 132 + x (16-byte writes of 512 contiguous bytes; the 64-bit reads of a half-warp,
    // 4 rows x 4 residues, fall on 16 distinct bank pairs)
    float2* const tb = R0 + warp_id * (32 * 34);
#pragma unroll
    for (int yl = 0; yl < 8; ++yl)
#pragma unroll
      for (int kk = 0; kk < 2; ++kk)
        *reinterpret_cast<float4*>(tb + yl * 132 + 64 * kk + 2 * lane_id) =
            make_float4(acc[yl * 4 + kk * 2].x, acc[yl * 4 + kk * 2].y, acc[yl * 4 + kk * 2 + 1].x,
                        acc[yl * 4 + kk * 2 + 1].y);
    __syncwarp();
    float2 v[32];
#pragma unroll
    for (int n1 = 0; n1 < 32; ++n1) v[n1] = tb[(lane_id >> 2) * 132 + 4 * n1 + (lane_id & 3)];
    __syncwarp();      // every lane has read its row before X1 overwrites the warp's rows
    // forward 2D DFT of Psi_p (passes A, B, C)
    passA_fwd(v, tA);
#pragma unroll
    for (int k = 0; k < 32; k += 2) x1w[k / 2] = make_float4(v[k].x, v[k].y, v[k + 1].x, v[k + 1].y);
    __syncthreads();
    float2 b0[16], b1[16];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        b0[q * 4 + r] = x1r[(128 * q + r) * 34];
        b1[q * 4 + r] = x1r[(128 * q + r) * 34 + 16];
      }
    passB_fwd(b0, tB);
    passB_fwd(b1, tB);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        x2b[(q * 4 + r) * 1024] = b0[q * 4 + r];
        x2b[(q * 4 + r) * 1024 + 16] = b1[q * 4 + r];
      }
    __syncthreads();
    const int warp = T >> 5, lane = T & 31;
    if constexpr (MODE == kReadAnnuli) {
      if (c_live) {
        float2 c[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) c[j] = x2c[j * 32];
        dft32<false>(c);
        // detector (Sec. 3.1, 2D STEM): sum of |DFT|^2 over the annulus
#pragma unroll
        for (int d = 0; d < kMaxDet; ++d) {
          if (d >= a.n_det) break;
          float sum = 0.f;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if ((dbits[d] >> j) & 1u) sum = fmaf(c[j].x, c[j].x, fmaf(c[j].y, c[j].y, sum));
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
          if (lane == 0) red[warp * kMaxDet + d] = sum;
        }
      } else if (lane < kMaxDet) {
        red[warp * kMaxDet + lane] = 0.f;
      }
      __syncthreads();
      if (T < a.n_det) {
        double tot = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) tot += static_cast<double>(red[w * kMaxDet + T]);
        a.acc[(static_cast<size_t>(a.cfg_base + cfg) * a.n_det + T) * a.n_probes + p] = tot * (1.0 / (kW * kW));
      }
    } else if constexpr (MODE == kReadLabels) {
      // 3D STEM (Sec. 3.1): |DFT|^2 into a W x W plane, then each label's pixels summed by
      // one warp in a fixed order (lane-strided partial sums, then a fixed shuffle tree)
      float e[32];
      if (c_live) {
        float2 c[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) c[j] = x2c[j * 32];
        dft32<false>(c);
#pragma unroll
        for (int j = 0; j < 32; ++j) e[j] = fmaf(c[j].x, c[j].x, c[j].y * c[j].y);
      }
      __syncthreads();   // every X2 read of R0 is done: R0 becomes the plane
      float* plane = reinterpret_cast<float*>(R0);
      if (c_live) {
#pragma unroll
        for (int j = 0; j < 32; ++j) plane[(k1y + 4 * j) * kW + kx] = e[j];
      }
      __syncthreads();
      for (int l = warp; l < a.n_det; l += kThreads / 32) {
        const int s0 = a.lab_start[l], s1 = a.lab_start[l + 1];
        float sum = 0.f;
        for (int i = s0 + lane; i < s1; i += 32) sum += plane[a.lab_pix[i]];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0)
          a.acc[(static_cast<size_t>(a.cfg_base + cfg) * a.n_det + l) * a.n_probes + p] =
              static_cast<double>(sum) * (1.0 / (kW * kW));
      }
    } else {
      // 4D STEM (Sec. 3.1): the pattern |DFT|^2 / W^2 on |kx| <= pat_a, |ky| <= pat_b, zero
      // outside the band, one FP32 slot per configuration
      const int pw = 2 * a.pat_a + 1;
      float* const out = a.pat + (static_cast<size_t>(cfg) * a.n_probes + p) * static_cast<size_t>(pw * (2 * a.pat_b + 1)) +
                         a.pat_b * pw + kxs + a.pat_a;
      const bool col = kxs >= -a.pat_a && kxs <= a.pat_a;
      if (c_live) {
        float2 c[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) c[j] = x2c[j * 32];
        dft32<false>(c);
        if (col) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int ky = k1y + 4 * j;
            const int kys = ky < 64 ? ky : ky - 128;
            if (kys >= -a.pat_b && kys <= a.pat_b)
              out[kys * pw] = kxs * kxs + kys * kys <= a.band_r2
                                  ? fmaf(c[j].x, c[j].x, c[j].y * c[j].y) * (1.f / (kW * kW))
                                  : 0.f;
          }
        }
      } else if (col) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int ky = k1y + 4 * j;
          const int kys = ky < 64 ? ky : ky - 128;
          if (kys >= -a.pat_b && kys <= a.pat_b) out[kys * pw] = 0.f;
        }
      }
    }
  }
}

// Step a4 for a group of neighbouring probes. The group's frame is the union of its probe
// windows: probe q = (qi, qj) of the group has its window at (qi psx, qj psy), and the
// translate of its entry j sits at that corner plus shift_j. The CTA sorts the group's
// entries by (translate, frame position, entry) in shared memory (bitonic sort, one entry per
// thread), merges equal (translate, position) pairs into one union entry u with a coefficient
// per probe (zero where the probe does not use it) and a mask of the probes that do.
// Each warp then takes blocks of 8 x 16 pixels of the frame: for every union entry whose
// window meets the block and that a probe covering the block uses, it loads the block's
// pixels once and adds them into the accumulators of all the group's probes (up to 4 probes
// x 4 pixels per lane), in union order, which for each probe is its ascending translate order;
// a zero coefficient leaves a sum unchanged. Pixels of a probe's accumulator outside that
// probe's window are never stored. The products are dense over the group (no per-probe
// branch): with groups of 16 probes and a branch per probe and entry the kernel spent most
// of its time on branches and instruction fetch.
template <bool HALF>
__global__ void __launch_bounds__(kThreads, 1) k_synth_group(const SynthArgs a, const GroupArgs g) {
  constexpr int kQ = kGroupDenseProbes, kE = kGroupMaxEntries;
  constexpr int kGQ = kGroupDenseProbes;   // accumulators per lane: every probe of the group
  static_assert(kE == kThreads, "one group entry per thread");
  extern __shared__ __align__(16) unsigned char smq[];
  uint64_t* const keys = reinterpret_cast<uint64_t*>(smq);                     // [kE]
  float4* const atab = reinterpret_cast<float4*>(keys + kE);                   // [u][q]: (ax, ax, -ay, ay)
  int4* const uent = reinterpret_cast<int4*>(atab + kE * kQ);                  // u: (x, y, probe mask, translate)
  int4* const pinfo = reinterpret_cast<int4*>(uent + kE);                      // probe q: (p, x0, y0)
  int* const wsum = reinterpret_cast<int*>(pinfo + kQ);                        // first entries per warp
  const int T = threadIdx.x, lane = T & 31, warp = T >> 5;
  const int W = a.W;
  const long long WW = static_cast<long long>(W) * W;
  const float2* const Uc = HALF ? nullptr : a.U + g.cfg * a.u_slot;
  const __half2* const Uhc = HALF ? static_cast<const __half2*>(a.Uh) + g.cfg * a.u_slot : nullptr;
  const float* const Usc = HALF ? a.Uscale + static_cast<size_t>(g.cfg) * a.n_translates : nullptr;
  const int r2 = lane >> 4, c16 = lane & 15;
  const int n_groups = g.ngx * g.ngy;
  const int p_base = g.gb_base * g.gy * a.npx;   // region index of psi's first probe
  for (int gi = blockIdx.x; gi < n_groups; gi += gridDim.x) {
    const int gid = probe_of(gi, g.ngx, g.ngy, g.gstrip);
    const int gl = gid / g.ngx, ga = gid - gl * g.ngx;
    const int a0 = ga * g.gx, b0 = (g.gb_base + gl) * g.gy;
    const int nqa = min(g.gx, a.npx - a0), nqb = min(g.gy, a.npy - b0);
    const int G = nqa * nqb, n_ent = G * a.L;
    __syncthreads();   // the previous group's reads of the tables are over
    {
      uint64_t key = ~0ull;
      if (T < n_ent) {
        const int q = T / a.L, j = T - q * a.L;
        const int qj = q / nqa, qi = q - qj * nqa;
        const size_t o = (static_cast<size_t>(b0 + qj) * a.npx + a0 + qi) * a.L + j;
        const int2 sh = a.shift[o];
        const uint64_t px = static_cast<uint64_t>(qi * g.psx + sh.x + kGroupPosBias);
        const uint64_t py = static_cast<uint64_t>(qj * g.psy + sh.y + kGroupPosBias);
        key = (static_cast<uint64_t>(a.tidx[o]) << 34) | (px << 22) | (py << 10) | static_cast<uint64_t>(T);
      }
      keys[T] = key;
      uent[T].z = 0;
#pragma unroll
      for (int q = 0; q < kQ; ++q) atab[q * kE + T] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (T < G) {
        const int qj = T / nqa, qi = T - qj * nqa;
        pinfo[T] = make_int4((b0 + qj) * a.npx + a0 + qi, qi * g.psx, qj * g.psy, 0);
      }
    }
    __syncthreads();
    for (int k = 2; k <= kE; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        const int l = T ^ j;
        if (l > T) {
          const uint64_t x = keys[T], y = keys[l];
          if ((x > y) == ((T & k) == 0)) {
            keys[T] = y;
            keys[l] = x;
          }
        }
        __syncthreads();
      }
    // union entries: the first of each run of equal (translate, position) keys
    const uint64_t kt = keys[T];
    const bool valid = T < n_ent;
    const bool first = valid && (T == 0 || (keys[T - 1] >> 10) != (kt >> 10));
    const uint32_t bal = __ballot_sync(0xffffffffu, first);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int before = 0, K = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) {
      const int c = wsum[w];
      before += w < warp ? c : 0;
      K += c;
    }
    if (valid) {
      const int u = before + __popc(bal & ((1u << lane) - 1u)) - (first ? 0 : 1);
      const int e = static_cast<int>(kt & 1023u);
      const int q = e / a.L, j = e - q * a.L;
      const int t = static_cast<int>(kt >> 34);
      float2 al = a.alpha[static_cast<size_t>(pinfo[q].x) * a.L + j];
      if constexpr (HALF) {
        const float f = Usc[t];
        al.x *= f;
        al.y *= f;
      }
      atab[u * kQ + q] = make_float4(al.x, al.x, -al.y, al.y);
      atomicOr(&uent[u].z, 1 << q);
      if (first) {
        uent[u].x = static_cast<int>((kt >> 22) & 4095u) - kGroupPosBias;
        uent[u].y = static_cast<int>((kt >> 10) & 4095u) - kGroupPosBias;
        uent[u].w = t;
      }
    }
    __syncthreads();
    // ---- the frame in blocks of 8 rows x 16 columns, one warp per block; lane (r, c) holds
    // rows r + 2 h (h < 4) of column c, for each of the group's (up to 4) probes
    const int Fx = (nqa - 1) * g.psx + kW, Fy = (nqb - 1) * g.psy + kW;
    const int nbx = (Fx + 15) >> 4, nblk = nbx * ((Fy + 7) >> 3);
    for (int bk = warp; bk < nblk; bk += kThreads / 32) {
      const int by0 = 8 * (bk / nbx), bx0 = 16 * (bk - (bk / nbx) * nbx);
      uint32_t cov = 0u;   // probes whose windows meet the block
      for (int q = 0; q < G; ++q) {
        const int4 pi = pinfo[q];
        if (bx0 < pi.y + kW && bx0 + 16 > pi.y && by0 < pi.z + kW && by0 + 8 > pi.z) cov |= 1u << q;
      }
      if (cov == 0u) continue;
      float2 acc[kGQ][4];
#pragma unroll
      for (int q = 0; q < kGQ; ++q)
#pragma unroll
        for (int h = 0; h < 4; ++h) acc[q][h] = make_float2(0.f, 0.f);
      // loads of two union entries (zero outside the translate's window; none for an entry
      // that no covering probe uses or whose window misses the block)
      auto fetch = [&](int u0, float2 (&v)[2][4], bool (&live)[2]) {
#pragma unroll
        for (int d = 0; d < 2; ++d) {
          const int u = u0 + d;
          live[d] = false;
#pragma unroll
          for (int h = 0; h < 4; ++h) v[d][h] = make_float2(0.f, 0.f);
          if (u < K) {
            const int4 E = uent[u];
            const int xw = bx0 - E.x, yw = by0 - E.y;   // the block's corner in the translate's window
            live[d] = xw < W && xw + 16 > 0 && yw < W && yw + 8 > 0 && (static_cast<uint32_t>(E.z) & cov) != 0u;
            if (live[d]) {
              const int x = xw + c16, y0 = yw + r2;
              const bool okx = static_cast<unsigned>(x) < static_cast<unsigned>(W);
              const long long tb = static_cast<long long>(E.w) * WW + x;
#pragma unroll
              for (int h = 0; h < 4; ++h) {
                const int y = y0 + 2 * h;
                if (okx && static_cast<unsigned>(y) < static_cast<unsigned>(W)) {
                  if constexpr (HALF)
                    v[d][h] = __half22float2(Uhc[tb + static_cast<long long>(y) * W]);
                  else
                    v[d][h] = Uc[tb + static_cast<long long>(y) * W];
                }
              }
            }
          }
        }
      };
      // their products into every probe's accumulator (a probe that does not use an entry
      // has a zero coefficient, which leaves its sums unchanged)
      auto consume = [&](int u0, const float2 (&v)[2][4], const bool (&live)[2]) {
#pragma unroll
        for (int d = 0; d < 2; ++d) {
          if (!live[d]) continue;
          const float4* const ar = atab + (u0 + d) * kQ;
          float4 al[kGQ];
#pragma unroll
          for (int q = 0; q < kGQ; ++q) al[q] = ar[q];
#pragma unroll
          for (int q = 0; q < kGQ; ++q)
#pragma unroll
            for (int h = 0; h < 4; ++h) acc[q][h] = cfma2(acc[q][h], al[q], v[d][h]);
        }
      };
      // two sets of loads in flight: the next two entries are fetched before the current two
      // are consumed
      float2 va[2][4], vb[2][4];
      bool la[2], lb[2];
      fetch(0, va, la);
      for (int u0 = 0; u0 < K; u0 += 4) {
        fetch(u0 + 2, vb, lb);
        consume(u0, va, la);
        fetch(u0 + 4, va, la);
        consume(u0 + 2, vb, lb);
      }
      // the block's pixels of each covering probe's window
#pragma unroll
      for (int q = 0; q < kGQ; ++q) {
        if (cov & (1u << q)) {
          const int4 pi = pinfo[q];
          const int lx = bx0 + c16 - pi.y, ly = by0 + r2 - pi.z;
          float2* const dst = g.psi + static_cast<size_t>(pi.x - p_base) * (kW * kW);
          if (static_cast<unsigned>(lx) < static_cast<unsigned>(kW)) {
#pragma unroll
            for (int h = 0; h < 4; ++h)
              if (static_cast<unsigned>(ly + 2 * h) < static_cast<unsigned>(kW))
                __stcs(dst + (ly + 2 * h) * kW + lx, acc[q][h]);
          }
        }
      }
    }
  }
}

__global__ void k_identity_tables(int n, int32_t* tidx, float2* alpha, int2* shift) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    tidx[i] = i;
    alpha[i] = make_float2(1.f, 0.f);
    shift[i] = make_int2(0, 0);
  }
}

__global__ void k_finalize_variants(const double* acc, int64_t n, int n_cfg, int n_var, const double* w,
                                    double* out) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double tot = 0.0;
  for (int v = 0; v < n_var; ++v) {
    double s = 0.0;
    for (int c = 0; c < n_cfg; ++c) s += acc[(static_cast<size_t>(v) * n_cfg + c) * n + i];
    tot += w[v] * s;
  }
  out[i] = tot;
}

__global__ void k_pattern_accumulate(const float* slots, int64_t n, int n_cfg, int first, double* acc) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = first ? 0.0 : acc[i];
  for (int c = 0; c < n_cfg; ++c) s += static_cast<double>(slots[static_cast<size_t>(c) * n + i]);
  acc[i] = s;
}

__global__ void k_pattern_finalize(const double* acc, int64_t n, double scale, float* out) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] = static_cast<float>(acc[i] * scale);
}

// ------------------------------------------------------------------------------------------
// step a1: potential and transmission
// ------------------------------------------------------------------------------------------
struct AtomRel {
  float x_hi, x_lo, y_hi, y_lo, peak;
};

// One CTA = a 16 x 16 pixel tile of one slice. Atoms of the slice are filtered
// against the tile in list order (ordered compaction), so every pixel adds its
// atom terms in the same order whatever the tile or rectangle: a partial
// rebuild is bitwise equal to a full one. Each pixel value is written to all
// its periodic copies in the padded array [ny + W][nx + W].
// Double-float arithmetic (an unevaluated sum h + l of two FP32 values): Knuth's two-sum is
// exact, so offsets of the FP64 atom positions from the tile centre stay accurate to about
// 2^-46 of their size with FP32 instructions only (FP64 runs at a small fraction of the FP32
// rate on this GPU).
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return make_float2(s, (a - (s - bb)) + (b - bb));
}
// (h + l) + (bh + bl), renormalized so that |l| <= ulp(h) / 2
__device__ __forceinline__ float2 df_add(float2 a, float bh, float bl) {
  const float2 s = two_sum(a.x, bh);
  const float e = s.y + (a.y + bl);
  const float h = s.x + e;
  return make_float2(h, e - (h - s.x));
}

// g (bh + bl) as hi + lo: g bh exactly as p + fma(g, bh, -p), plus g bl
__device__ __forceinline__ float2 prod_df(float g, float bh, float bl) {
  const float p = g * bh;
  const float e = fmaf(g, bl, fmaf(g, bh, -p));
  const float h = p + e;
  return make_float2(h, e - (h - p));
}

__global__ void __launch_bounds__(256) k_potential(const PotArgs a) {
  __shared__ AtomRel lst[256];
  __shared__ int wcount[8];
  const int s = blockIdx.z;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int bx = blockIdx.x * 16, by = blockIdx.y * 16;
  const bool in_rect = (bx + tx < a.rw) && (by + ty < a.rh);
  const int gx0 = (a.rx0 + bx) % a.nx;
  const int gy0 = (a.ry0 + by) % a.ny;
  // atoms are taken relative to the tile centre (gx0 + 7.5) dx, formed as hi + lo from the
  // pair dx = dx_hi + dx_lo with an exact FMA product (gx0 + 7.5 is exact in FP32)
  const float2 xc = prod_df(static_cast<float>(gx0) + 7.5f, a.dx_hi, a.dx_lo);
  const float2 yc = prod_df(static_cast<float>(gy0) + 7.5f, a.dy_hi, a.dy_lo);
  const float xch = xc.x, xcl = xc.y, ych = yc.x, ycl = yc.y;
  const float hlx = 0.5f * a.lx_hi, hly = 0.5f * a.ly_hi;
  const int a0 = a.slice_start[s], a1 = a.slice_start[s + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float v = 0.f;
  for (int base = a0; base < a1; base += 256) {
    const int k = base + threadIdx.x;
    bool keep = false;
    AtomRel e{0.f, 0.f, 0.f, 0.f, 0.f};
    if (k < a1) {
      // positions lie in [0, l) and the tile centre in [0, l + 8 dx): one period at most
      // brings the offset to its minimum image (decided on the high part: an offset near
      // half a period is far outside the tile either way)
      float2 ddx = df_add(a.ax[k], -xch, -xcl), ddy = df_add(a.ay[k], -ych, -ycl);
      if (ddx.x >= hlx)
        ddx = df_add(ddx, -a.lx_hi, -a.lx_lo);
      else if (ddx.x < -hlx)
        ddx = df_add(ddx, a.lx_hi, a.lx_lo);
      if (ddy.x >= hly)
        ddy = df_add(ddy, -a.ly_hi, -a.ly_lo);
      else if (ddy.x < -hly)
        ddy = df_add(ddy, a.ly_hi, a.ly_lo);
      keep = fabsf(ddx.x) < a.limx && fabsf(ddy.x) < a.limy;
      if (keep) {
        // offset from pixel (0, 0) of the tile, as hi + lo
        const float2 rx = df_add(ddx, a.c75x_hi, a.c75x_lo), ry = df_add(ddy, a.c75y_hi, a.c75y_lo);
        e.x_hi = rx.x;
        e.x_lo = rx.y;
        e.y_hi = ry.x;
        e.y_lo = ry.y;
        const int spc = a.asp[k];
        e.peak = (spc >= 0 && spc < a.n_species) ? a.peak[spc] : 0.f;
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) wcount[warp] = __popc(bal);
    __syncthreads();
    int off = 0, total = 0;
    for (int w = 0; w < 8; ++w) {
      off += (w < warp) ? wcount[w] : 0;
      total += wcount[w];
    }
    if (keep) lst[off + __popc(bal & ((1u << lane) - 1u))] = e;
    __syncthreads();
    for (int j = 0; j < total; ++j) {
      const AtomRel at = lst[j];
      const float ddx = fmaf(static_cast<float>(tx), a.dx_hi, -at.x_hi) +
                        fmaf(static_cast<float>(tx), a.dx_lo, -at.x_lo);
      const float ddy = fmaf(static_cast<float>(ty), a.dy_hi, -at.y_hi) +
                        fmaf(static_cast<float>(ty), a.dy_lo, -at.y_lo);
      const float r2 = ddx * ddx + ddy * ddy;
      if (r2 < a.rc2) {
        float g = 0.f;
        for (int q = 0; q < a.n_terms; ++q) g = fmaf(a.frac[q], expf(-r2 * a.inv2w2[q]), g);
        v = fmaf(at.peak, g, v);
      }
    }
    __syncthreads();
  }
  if (in_rect) {
    int gx = gx0 + tx;
    if (gx >= a.nx) gx -= a.nx;
    int gy = gy0 + ty;
    if (gy >= a.ny) gy -= a.ny;
    float sn, cs;
    sincosf(a.sigma * v, &sn, &cs);
    const float2 tv = make_float2(cs, sn);
    const int pitch = a.nx + kW;
    float2* ts = a.t + static_cast<size_t>(s) * pitch * (a.ny + kW);
    ts[static_cast<size_t>(gy) * pitch + gx] = tv;
    const bool hx = gx < kW, hy = gy < kW;
    if (hx) ts[static_cast<size_t>(gy) * pitch + gx + a.nx] = tv;
    if (hy) ts[static_cast<size_t>(gy + a.ny) * pitch + gx] = tv;
    if (hx && hy) ts[static_cast<size_t>(gy + a.ny) * pitch + gx + a.nx] = tv;
  }
}

__global__ void k_expand_half(const __half2* src, float scale, float2* dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kW * kW) {
    const float2 u = __half22float2(src[i]);
    dst[i] = make_float2(u.x * scale, u.y * scale);
  }
}

// step a6: average over configurations, summed in configuration order (deterministic)
__global__ void k_finalize(const double* acc, int64_t n, int n_cfg, double scale, double* out) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) {
    double s = 0.0;
    for (int c = 0; c < n_cfg; ++c) s += acc[static_cast<size_t>(c) * n + i];
    out[i] = s * scale;
  }
}

// ------------------------------------------------------------------------------------------
// scratch of the no-allocation readout
// ------------------------------------------------------------------------------------------
// One file-scope array on every device that loads this library, held until the
// process exits. lma_readout_noalloc places its per-call tables and its FP64
// accumulator here instead of allocating. Host code must not use the symbol's
// name as an address: noalloc_scratch() looks the device address up with
// cudaGetSymbolAddress, once per device, with that device current.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

cudaError_t noalloc_scratch(void** ptr) {
  static std::mutex mu;
  static void* addr[kMaxDevices] = {};
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    addr[dev] = p;
  }
  *ptr = addr[dev];
  return cudaSuccess;
}

// ------------------------------------------------------------------------------------------
// host-side launchers
// ------------------------------------------------------------------------------------------
size_t slice_smem_bytes() { return static_cast<size_t>(kSliceSmemFloat2) * sizeof(float2); }
size_t synth_smem_bytes() { return static_cast<size_t>(kSynthSmemFloat2) * sizeof(float2); }
size_t slice_tc_smem_bytes() { return static_cast<size_t>(kSliceTcSmemBytes); }
static size_t slice_gen_smem_bytes(int W) {
  return W <= 64 ? (3 * static_cast<size_t>(w64::kBufE) + w64::kN) * sizeof(float2)   // A, B, staged t, ey
                 : (2 * static_cast<size_t>(w256::kBuf) + w256::kN) * sizeof(float2) +
                       (2 + 2 * gen::kThreadsGen / 32) * sizeof(uint64_t);   // two panel buffers, ey, mbarriers
}
cudaError_t launch_selftest_wait(int which, int* status, cudaStream_t s) {
  k_selftest_wait<<<1, which == 0 ? 32 : gen::kThreadsGen, 0, s>>>(status);
  return cudaGetLastError();
}
size_t slice_gen_scratch_bytes(int W) {
  return W <= 64 ? 0 : static_cast<size_t>(sm_count()) * W * W * sizeof(float2);
}
size_t slice_rs_smem_bytes() { return static_cast<size_t>(kW * kW + 32 * 32) * sizeof(float2); }

cudaError_t init_device_constants() {
  float2 w[128];
  const double pi = 3.14159265358979323846;
  for (int m = 0; m < 128; ++m) {
    const double ang = -2.0 * pi * m / 128.0;
    w[m] = make_float2(static_cast<float>(cos(ang)), static_cast<float>(sin(ang)));
  }
  cudaError_t e = cudaMemcpyToSymbol(c_w128, w, sizeof(w));
  if (e != cudaSuccess) return e;
  float2 tt[16];
  for (int m = 0; m < 16; ++m) {
    const double th = 2.0 * pi * m / 32.0, c = cos(th), sn = sin(th);
    tt[m] = (m <= 4 || m >= 12) ? make_float2(static_cast<float>(c), static_cast<float>(sn / c))
                                : make_float2(static_cast<float>(sn), static_cast<float>(c / sn));
  }
  e = cudaMemcpyToSymbol(c_tw32t, tt, sizeof(tt));
  if (e != cudaSuccess) return e;
  float4 ra[32], rb[32];
  for (int k1 = 0; k1 < 32; ++k1) {
    double sc[4] = {1, 0, 0, 0}, t[4] = {0, 0, 0, 0};
    for (int r = 1; r <= 3; ++r) {
      // forward W_128^(r k1) = (cos th, -sin th) = s (1, t) or s (t, 1)
      const double th = 2.0 * pi * r * k1 / 128.0, c = cos(th), sn = sin(th);
      if (k1 < 16) {
        sc[r] = c;
        t[r] = -sn / c;
      } else {
        sc[r] = -sn;
        t[r] = c / -sn;
      }
    }
    ra[k1] = make_float4(static_cast<float>(t[1]), static_cast<float>(sc[1]), static_cast<float>(t[2]),
                         static_cast<float>(sc[2]));
    rb[k1] = make_float4(static_cast<float>(t[3]), static_cast<float>(sc[3]), static_cast<float>(sc[3] / sc[1]), 0.f);
  }
  if ((e = cudaMemcpyToSymbol(c_twrA, ra, sizeof(ra))) != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_twrB, rb, sizeof(rb));
  if (e != cudaSuccess) return e;
  const int ss = static_cast<int>(slice_smem_bytes()), sy = static_cast<int>(synth_smem_bytes());
  {
    const void* ks[8] = {reinterpret_cast<const void*>(k_slice<false, false, false>), reinterpret_cast<const void*>(k_slice<false, false, true>),
                         reinterpret_cast<const void*>(k_slice<false, true, false>),  reinterpret_cast<const void*>(k_slice<false, true, true>),
                         reinterpret_cast<const void*>(k_slice<true, false, false>),  reinterpret_cast<const void*>(k_slice<true, false, true>),
                         reinterpret_cast<const void*>(k_slice<true, true, false>),   reinterpret_cast<const void*>(k_slice<true, true, true>)};
    for (const void* f : ks)
      if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, ss)) != cudaSuccess) return e;
  }
  {
    // B^T[n][k] of the 32-point DFT in real form (n: output column of [Re y | Im y], k: input
    // of [Re x | Im x]; F[k][n] = exp(-2 pi i k n / 32)), split into FP16 high and low parts;
    // then the same for conj F (the inverse): the off-diagonal blocks change sign
    std::vector<unsigned char> bt(4 * tc::kBBytes, 0);
    for (int inv = 0; inv < 2; ++inv)
      for (int n = 0; n < 64; ++n)
        for (int k = 0; k < 64; ++k) {
          const int kk = k & 31, nn = n & 31;
          const double th = 2.0 * pi * ((kk * nn) & 31) / 32.0;
          const double fr = cos(th), fi = inv ? sin(th) : -sin(th);
          const double val = n < 32 ? (k < 32 ? fr : -fi) : (k < 32 ? fi : fr);
          const __half hi = __float2half_rn(static_cast<float>(val));
          const __half lo = __float2half_rn(static_cast<float>(val - static_cast<double>(__half2float(hi))));
          const size_t base = static_cast<size_t>(inv) * 2 * tc::kBBytes;
          std::memcpy(&bt[base + tc::op_offset(n, k)], &hi, 2);
          std::memcpy(&bt[base + tc::kBBytes + tc::op_offset(n, k)], &lo, 2);
        }
    if ((e = cudaMemcpyToSymbol(g_tc_dft32, bt.data(), bt.size())) != cudaSuccess) return e;
    const int st = static_cast<int>(slice_tc_smem_bytes());
    for (auto f : {k_slice_tc<false, false>, k_slice_tc<false, true>, k_slice_tc<true, false>, k_slice_tc<true, true>})
      if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, st)) != cudaSuccess) return e;
  }
  {
    // twiddles of the W = 64 and W = 256 transforms: exp(-2 pi i m / W), m < W
    float2 tw1[w64::kN];
    for (int m = 0; m < w64::kN; ++m)
      tw1[m] = make_float2(static_cast<float>(cos(-2.0 * pi * m / 64)), static_cast<float>(sin(-2.0 * pi * m / 64)));
    if ((e = cudaMemcpyToSymbol(w64::c_tw, tw1, sizeof(tw1))) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_slice_64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(slice_gen_smem_bytes(64)))) != cudaSuccess)
      return e;
    float2 tw2[w256::kN];
    for (int m = 0; m < w256::kN; ++m)
      tw2[m] = make_float2(static_cast<float>(cos(-2.0 * pi * m / 256)), static_cast<float>(sin(-2.0 * pi * m / 256)));
    if ((e = cudaMemcpyToSymbol(w256::c_tw, tw2, sizeof(tw2))) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_slice_256, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(slice_gen_smem_bytes(256)))) != cudaSuccess)
      return e;
  }
  const int sr = static_cast<int>(slice_rs_smem_bytes());
  for (auto f : {k_slice_rs<3, 4, 3>, k_slice_rs<5, 4, 5>, k_slice_rs<3, 4>, k_slice_rs<5, 4>, k_slice_rs<7, 2>, k_slice_rs<9, 2>, k_slice_rs<11, 2>,
                 k_slice_rs<13, 2>, k_slice_rs<15, 2>, k_slice_rs<17, 2>, k_slice_rs<19, 2>, k_slice_rs<21, 2>,
                 k_slice_rs<23, 2>, k_slice_rs<25, 2>})
    if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, sr)) != cudaSuccess) return e;
  for (auto f : {k_synth_detect<false, kReadAnnuli, false>, k_synth_detect<true, kReadAnnuli, false>,
                 k_synth_detect<false, kReadLabels, false>, k_synth_detect<true, kReadLabels, false>,
                 k_synth_detect<false, kReadPattern, false>, k_synth_detect<true, kReadPattern, false>,
                 k_synth_detect<false, kReadAnnuli, true>, k_synth_detect<true, kReadAnnuli, true>,
                 k_synth_detect<false, kReadLabels, true>, k_synth_detect<true, kReadLabels, true>,
                 k_synth_detect<false, kReadPattern, true>, k_synth_detect<true, kReadPattern, true>,
                 k_synth_detect<false, kReadAnnuli, false, 0>, k_synth_detect<false, kReadLabels, false, 0>,
                 k_synth_detect<false, kReadPattern, false, 0>})
    if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, sy)) != cudaSuccess) return e;
  for (auto f : {k_synth_group<false>, k_synth_group<true>})
    if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(synth_group_smem_bytes()))) != cudaSuccess)
      return e;
  return cudaSuccess;
}

cudaError_t launch_potential(const PotArgs& a, cudaStream_t s) {
  dim3 grid((a.rw + 15) / 16, (a.rh + 15) / 16, a.n_slices);
  k_potential<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      n = v;
    else
      return 1;
  }
  return n;
}

cudaError_t launch_slice(const SliceLaunch& a, bool even_origins, bool half, int mode, cudaStream_t s) {
  if (a.n_list <= 0) return cudaSuccess;
  if (a.n_jobs < 1 || a.n_jobs > kMaxJobs || a.start[0] != 0 || a.start[a.n_jobs] != a.n_list)
    return cudaErrorInvalidValue;
  if (mode == kSliceDynamic && !a.counter) return cudaErrorInvalidValue;
  const size_t sm = slice_smem_bytes();
  // one CTA per SM fits (216 KiB of shared memory): persistent grids are one wave
  const int grid = mode == kSliceOnePerItem ? a.n_list : (a.n_list < sm_count() ? a.n_list : sm_count());
  if (mode == kSliceDynamic) {
    cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
  }
  // the pruned kernel needs every job's bandlimit radius below 44 pixels (|ky| >= 44 for
  // pass C's entries 11..20; |kx| >= 48 for pass B's masked columns)
  bool prune = true;
  for (int i = 0; i < a.n_jobs; ++i) prune = prune && a.job[i].r2max < 44 * 44;
  using K = void (*)(const SliceLaunch, const int);
  static const K table[8] = {k_slice<false, false, false>, k_slice<false, false, true>, k_slice<false, true, false>,
                             k_slice<false, true, true>,   k_slice<true, false, false>,  k_slice<true, false, true>,
                             k_slice<true, true, false>,   k_slice<true, true, true>};
  const K f = table[(even_origins ? 4 : 0) + (half ? 2 : 0) + (prune ? 1 : 0)];
  f<<<grid, kThreads, sm, s>>>(a, mode);
  return cudaGetLastError();
}

cudaError_t launch_slice_tc(const SliceLaunch& a, bool even_origins, cudaStream_t s) {
  if (a.n_list <= 0) return cudaSuccess;
  if (a.n_jobs < 1 || a.n_jobs > kMaxJobs || a.start[0] != 0 || a.start[a.n_jobs] != a.n_list || !a.status)
    return cudaErrorInvalidValue;
  bool prune = true;
  for (int i = 0; i < a.n_jobs; ++i) prune = prune && a.job[i].r2max < 44 * 44;
  // persistent: one CTA per SM (its shared memory admits no second one), which holds the
  // 256 TMEM columns it allocates for the whole launch
  const int grid = a.n_list < sm_count() ? a.n_list : sm_count();
  const size_t sm = slice_tc_smem_bytes();
  using K = void (*)(const SliceLaunch, int*);
  static const K table[4] = {k_slice_tc<false, false>, k_slice_tc<false, true>, k_slice_tc<true, false>,
                             k_slice_tc<true, true>};
  table[(even_origins ? 2 : 0) + (prune ? 1 : 0)]<<<grid, kThreads, sm, s>>>(a, a.status);
  return cudaGetLastError();
}

cudaError_t launch_slice_gen(const SliceLaunch& a, int W, float2* scratch, cudaStream_t s) {
  if (a.n_list <= 0) return cudaSuccess;
  if (a.n_jobs < 1 || a.n_jobs > kMaxJobs || a.start[0] != 0 || a.start[a.n_jobs] != a.n_list || !a.status)
    return cudaErrorInvalidValue;
  // persistent, one CTA per SM: W = 256 takes one scratch wave per CTA
  const int grid = a.n_list < sm_count() ? a.n_list : sm_count();
  if (W == 64) {
    // two CTAs per SM
    const int grid64 = a.n_list < 2 * sm_count() ? a.n_list : 2 * sm_count();
    k_slice_64<<<grid64, 512, slice_gen_smem_bytes(64), s>>>(a);
  } else if (W == 256) {
    if (!scratch) return cudaErrorInvalidValue;
    k_slice_256<<<grid, gen::kThreadsGen, slice_gen_smem_bytes(256), s>>>(a, scratch, a.status);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_slice_rs(const SliceLaunch& a, const float2* q, int K1, int K2, cudaStream_t s) {
  if (a.n_list <= 0) return cudaSuccess;
  if (K2 < 1 || K2 > 25 || (K2 & 1) == 0) return cudaErrorInvalidValue;
  const size_t sm = slice_rs_smem_bytes();
  switch (K1) {
    case 3:
      if (K2 == 3) k_slice_rs<3, 4, 3><<<a.n_list, kThreads, sm, s>>>(a, q, K2);
      else k_slice_rs<3, 4><<<a.n_list, kThreads, sm, s>>>(a, q, K2);
      break;
    case 5:
      if (K2 == 5) k_slice_rs<5, 4, 5><<<a.n_list, kThreads, sm, s>>>(a, q, K2);
      else k_slice_rs<5, 4><<<a.n_list, kThreads, sm, s>>>(a, q, K2);
      break;
    case 7: k_slice_rs<7, 2><<<a.n_list, kThreads, sm, s>>>(a, q, K2); break;
    case 9: k_slice_rs<9, 2><<<a.n_list, kThreads, sm, s>>>(a, q, K2); break;
    case 11: k_slice_rs<11, 2><<<a.n_list, kThreads, sm, s>>>(a, q, K2); break;
    case 13: k_slice_rs<13, 2><<<a.n_list, kThreads, sm, s>>>(a, q, K2); break;
    case 15: k_slice_rs<15, 2><<<a.n_list, kThreads, sm, s>>>(a, q, K2); break;
    case 17: k_slice_rs<17, 2><<<a.n_list, kThreads, sm, s>>>(a, q, K2); break;
    case 19: k_slice_rs<19, 2><<<a.n_list, kThreads, sm, s>>>(a, q, K2); break;
    case 21: k_slice_rs<21, 2><<<a.n_list, kThreads, sm, s>>>(a, q, K2); break;
    case 23: k_slice_rs<23, 2><<<a.n_list, kThreads, sm, s>>>(a, q, K2); break;
    case 25: k_slice_rs<25, 2><<<a.n_list, kThreads, sm, s>>>(a, q, K2); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_synth(const SynthArgs& a, bool half, int mode, int grid_mode, cudaStream_t s) {
  const int n_walk = a.probe_list ? a.n_list : a.n_probes;
  if (n_walk <= 0) return cudaSuccess;
  // kSynthGridAuto: the complex64 store persistent, one CTA per SM walking the items in order
  // (the per-CTA set-up is paid once; 30.5 -> 29.7 ms on the benchmark), the FP16 store one
  // CTA per item, whose hardware scheduling balances its shorter items better (28.1 ms against
  // 31.6 persistent); the other modes force one of the two (the autotuner times both)
  const int n_items = n_walk * a.n_cfg;
  const bool persistent = grid_mode == kSynthGridPersistent || (grid_mode == kSynthGridAuto && !half);
  const int grid = persistent ? (n_items < sm_count() ? n_items : sm_count()) : n_items;
  const size_t sm = synth_smem_bytes();
  // periodic probe windows (the window is the whole cell) wrap; others are zero outside
  using K = void (*)(const SynthArgs);
  static const K table[2][3][2] = {
      {{k_synth_detect<false, kReadAnnuli, false>, k_synth_detect<false, kReadAnnuli, true>},
       {k_synth_detect<false, kReadLabels, false>, k_synth_detect<false, kReadLabels, true>},
       {k_synth_detect<false, kReadPattern, false>, k_synth_detect<false, kReadPattern, true>}},
      {{k_synth_detect<true, kReadAnnuli, false>, k_synth_detect<true, kReadAnnuli, true>},
       {k_synth_detect<true, kReadLabels, false>, k_synth_detect<true, kReadLabels, true>},
       {k_synth_detect<true, kReadPattern, false>, k_synth_detect<true, kReadPattern, true>}}};
  if (mode != kReadAnnuli && mode != kReadLabels && mode != kReadPattern) return cudaErrorInvalidValue;
  const int mi = mode == kReadAnnuli ? 0 : (mode == kReadLabels ? 1 : 2);
  if (a.W != kW) {
    // other windows: complex64 store, non-periodic placement, W read at run time
    static const K other[3] = {k_synth_detect<false, kReadAnnuli, false, 0>, k_synth_detect<false, kReadLabels, false, 0>,
                               k_synth_detect<false, kReadPattern, false, 0>};
    if (half || a.cyclic || a.W < 32 || a.W > 256) return cudaErrorInvalidValue;
    other[mi]<<<grid, kThreads, sm, s>>>(a);
    return cudaGetLastError();
  }
  table[half ? 1 : 0][mi][a.cyclic ? 1 : 0]<<<grid, kThreads, sm, s>>>(a);
  return cudaGetLastError();
}

size_t synth_group_smem_bytes() {
  return static_cast<size_t>(kGroupMaxEntries) * (8 + 16 * kGroupDenseProbes + 16) + 16 * kGroupDenseProbes +
         4 * (kThreads / 32);
}

cudaError_t launch_synth_group(const SynthArgs& a, const GroupArgs& g, bool half, int grid_mode, cudaStream_t s) {
  const int n_groups = g.ngx * g.ngy;
  if (n_groups <= 0) return cudaSuccess;
  if (a.probe_list || a.cyclic || a.L < 1 || g.gx < 1 || g.gy < 1 || g.gx * g.gy > kGroupDenseProbes ||
      g.gx * g.gy * a.L > kGroupMaxEntries || (half && a.W != kW) || a.W < 32 || a.W > 256 || !g.psi)
    return cudaErrorInvalidValue;
  const int grid = grid_mode == kSynthGridPerItem ? n_groups : (n_groups < sm_count() ? n_groups : sm_count());
  const size_t sm = synth_group_smem_bytes();
  if (half)
    k_synth_group<true><<<grid, kThreads, sm, s>>>(a, g);
  else
    k_synth_group<false><<<grid, kThreads, sm, s>>>(a, g);
  return cudaGetLastError();
}

cudaError_t launch_identity_tables(int n, int32_t* tidx, float2* alpha, int2* shift, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_identity_tables<<<(n + 255) / 256, 256, 0, s>>>(n, tidx, alpha, shift);
  return cudaGetLastError();
}

cudaError_t launch_finalize_variants(const double* acc, int64_t n, int n_cfg, int n_var, const double* w, double* out,
                                     cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_finalize_variants<<<static_cast<int>((n + 255) / 256), 256, 0, s>>>(acc, n, n_cfg, n_var, w, out);
  return cudaGetLastError();
}

cudaError_t launch_pattern_accumulate(const float* slots, int64_t n, int n_cfg, bool first, double* acc,
                                      cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_pattern_accumulate<<<static_cast<int>((n + 255) / 256), 256, 0, s>>>(slots, n, n_cfg, first ? 1 : 0, acc);
  return cudaGetLastError();
}

cudaError_t launch_pattern_finalize(const double* acc, int64_t n, double scale, float* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_pattern_finalize<<<static_cast<int>((n + 255) / 256), 256, 0, s>>>(acc, n, scale, out);
  return cudaGetLastError();
}

cudaError_t launch_expand_half(const void* src, float scale, float2* dst, cudaStream_t s) {
  k_expand_half<<<(kW * kW + 255) / 256, 256, 0, s>>>(static_cast<const __half2*>(src), scale, dst);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const double* acc, int64_t n, int n_cfg, double scale, double* out,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int blocks = static_cast<int>((n + 255) / 256);
  k_finalize<<<blocks, 256, 0, s>>>(acc, n, n_cfg, scale, out);
  return cudaGetLastError();
}

}  // namespace lma_dev
