// common.cuh - device building blocks shared by the libbltt kernels: complex arithmetic in FP64,
// FP32 and double-float (an FP64-accurate number carried as an unevaluated sum of two FP32 values,
// run on the FP32 pipes), the shared-memory Stockham FFT engine and block reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "convert.cuh"

namespace bltt {

// log2 of a power of two, at compile time
__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v >> 1); }

// ------------------------------------------------------------------------------------------
// complex numbers as CUDA vector types
template <typename T> struct cplx;
template <> struct cplx<double> { using t = double2; };
template <> struct cplx<float> { using t = float2; };
template <typename T> using C = typename cplx<T>::t;
template <typename T> __device__ __forceinline__ C<T> mk(T re, T im) { C<T> r; r.x = re; r.y = im; return r; }

// ------------------------------------------------------------------------------------------
// double-float scalars: value = hi + lo with |lo| <= ulp(hi)/2.  The error-free transforms use
// the _rn intrinsics so that the compiler never fuses them into FMAs.
struct dfl {
  float hi, lo;
};

// double <-> double-float: the FP32 parts are converted on the integer pipes.  double -> pair:
// hi = x rounded to FP32; lo = x - hi rounded to FP32.  x - hi is the mantissa remainder below
// hi's 24 bits, an integer r (|r| <= 2^28) times 2^(E-1075), so lo is the rounded integer times
// that power of two, which equals the rounded FP64 difference whenever the power of two and lo
// are normal FP32 numbers (949 <= E <= 1149); other exponents take the FP64 subtraction.
// pair -> double leaves one FP64 addition.
__device__ __forceinline__ dfl df_from(double x) {
  const uint64_t b = bits_d(x);
  const uint32_t hw = (uint32_t)(b >> 32), lw = (uint32_t)b;
  const int E = (int)((hw >> 20) & 0x7FFu);
  if (E < 949 || E > 1149) {
    const float h = d2f_bits(x);
    return {h, d2f_bits(x - f2d_bits(h))};
  }
  const uint32_t sign = hw & 0x80000000u;
  const uint32_t m = ((hw & 0xFFFFFu) << 3) | (lw >> 29);       // top 23 mantissa bits
  const uint32_t rest = lw & 0x1FFFFFFFu;                        // 29 dropped bits
  const uint32_t up = (rest > 0x10000000u) | ((rest == 0x10000000u) & (m & 1u));
  const float h = __uint_as_float(((((uint32_t)(E - 1023 + 127)) << 23) + m + up) | sign);
  const int r = (int)rest - (int)(up << 29);                     // x - h in units of 2^(E-1075)
  const float lm = __int2float_rn(r) * __uint_as_float((uint32_t)(E - 1075 + 127) << 23);
  return {h, __uint_as_float(__float_as_uint(lm) ^ (r != 0 ? sign : 0u))};
}
__device__ __forceinline__ double df_to(dfl a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }
__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }

// a + b: two-sum of the leading parts, the trailing parts added once, then renormalised
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  float s = __fadd_rn(a.hi, b.hi);
  float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }

// a + b without the final renormalisation: (s, e) with s = fl(a.hi + b.hi) and e its exact error
// plus the trailing parts.  The pair still represents the sum to the same accuracy; |e| may reach
// a few ulp(s), which costs about one bit in the next operation.  For intermediate sums whose
// next use is another addition or multiplication.
__device__ __forceinline__ dfl df_add_nr(dfl a, dfl b) {
  float s = __fadd_rn(a.hi, b.hi);
  float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return {s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
}
__device__ __forceinline__ dfl df_sub_nr(dfl a, dfl b) { return df_add_nr(a, df_neg(b)); }

// a * b: exact product of the leading parts by FMA, cross terms folded into the error
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float h = __fadd_rn(p, e);
  return {h, __fsub_rn(e, __fsub_rn(h, p))};
}

// a * b without the final renormalisation (see df_add_nr)
__device__ __forceinline__ dfl df_mul_nr(dfl a, dfl b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return {p, e};
}

// a * b + c * d with one renormalisation
__device__ __forceinline__ dfl df_dot2(dfl a, dfl b, dfl c, dfl d) {
  float p1 = __fmul_rn(a.hi, b.hi);
  float e1 = __fmaf_rn(a.hi, b.hi, -p1);
  float p2 = __fmul_rn(c.hi, d.hi);
  float e2 = __fmaf_rn(c.hi, d.hi, -p2);
  float s = __fadd_rn(p1, p2);
  float bb = __fsub_rn(s, p1);
  float es = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bb)), __fsub_rn(p2, bb));
  float err = __fadd_rn(__fadd_rn(e1, e2), es);
  err = __fmaf_rn(a.hi, b.lo, err);
  err = __fmaf_rn(a.lo, b.hi, err);
  err = __fmaf_rn(c.hi, d.lo, err);
  err = __fmaf_rn(c.lo, d.hi, err);
  float h = __fadd_rn(s, err);
  return {h, __fsub_rn(err, __fsub_rn(h, s))};
}

// a * b + c * d without the final renormalisation (see df_add_nr)
__device__ __forceinline__ dfl df_dot2_nr(dfl a, dfl b, dfl c, dfl d) {
  float p1 = __fmul_rn(a.hi, b.hi);
  float e1 = __fmaf_rn(a.hi, b.hi, -p1);
  float p2 = __fmul_rn(c.hi, d.hi);
  float e2 = __fmaf_rn(c.hi, d.hi, -p2);
  float s = __fadd_rn(p1, p2);
  float bb = __fsub_rn(s, p1);
  float es = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bb)), __fsub_rn(p2, bb));
  float err = __fadd_rn(__fadd_rn(e1, e2), es);
  err = __fmaf_rn(a.hi, b.lo, err);
  err = __fmaf_rn(a.lo, b.hi, err);
  err = __fmaf_rn(c.hi, d.lo, err);
  err = __fmaf_rn(c.lo, d.hi, err);
  return {s, err};
}

// ------------------------------------------------------------------------------------------
// Arithmetic traits of the FFT engine.  V: a complex value; R: its real scalar.
struct ArithD {
  using V = double2;
  using R = double;
  using Sc = double;   // real scale factor
  static __device__ __forceinline__ Sc make_sc(double s) { return s; }
  static __device__ __forceinline__ Sc row_sc(const double* t64, const float*, int p) { return t64[p]; }
  static __device__ __forceinline__ V scale_sc(V a, Sc s) { return make_double2(a.x * s, a.y * s); }
  static __device__ __forceinline__ Sc neg_imag_sc(V a) { return -a.y; }   // -Im a as a scale
  static __device__ __forceinline__ double part_sc(V a, int comp, Sc s) { return (comp ? a.y : a.x) * s; }
  static __device__ __forceinline__ void put_sc(V* buf, int idx, int comp, double x, Sc s) {
    reinterpret_cast<double*>(buf)[2 * idx + comp] = x * s;
  }
  static __device__ __forceinline__ void put_sc2(V* buf, int i1, int i2, int comp, double x, Sc s) {
    const double v = x * s;
    reinterpret_cast<double*>(buf)[2 * i1 + comp] = v;
    reinterpret_cast<double*>(buf)[2 * i2 + comp] = v;
  }
  static __device__ __forceinline__ V add(V a, V b) { return make_double2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ V sub(V a, V b) { return make_double2(a.x - b.x, a.y - b.y); }
  static __device__ __forceinline__ V add_nr(V a, V b) { return add(a, b); }
  static __device__ __forceinline__ V sub_nr(V a, V b) { return sub(a, b); }
  static __device__ __forceinline__ V conj(V a) { return make_double2(a.x, -a.y); }
  static __device__ __forceinline__ V mul(V a, V b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
  }
  static __device__ __forceinline__ V mulc(V a, V b) {   // a * conj(b)
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
  }
  static __device__ __forceinline__ V mul_nr(V a, V b) { return mul(a, b); }
  static __device__ __forceinline__ V mulc_nr(V a, V b) { return mulc(a, b); }
  template <bool INV> static __device__ __forceinline__ V rot(V a) {   // * -i (fwd), * i (inv)
    return INV ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x);
  }
  static __device__ __forceinline__ V scale(V a, double s) { return make_double2(a.x * s, a.y * s); }
  static __device__ __forceinline__ V zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ V from(double re, double im) { return make_double2(re, im); }
  // a compile-time constant given in FP64 and as FP32 leading + trailing parts
  static __device__ __forceinline__ V cst(double re, double im, float, float, float, float) {
    return make_double2(re, im);
  }
  static __device__ __forceinline__ double part(V a, int comp) { return comp ? a.y : a.x; }
  static __device__ __forceinline__ void put(V* buf, int idx, int comp, double x) {
    reinterpret_cast<double*>(buf)[2 * idx + comp] = x;
  }
  static __device__ __forceinline__ void put_pm(V* buf, int i1, int i2, int comp, double x) {
    reinterpret_cast<double*>(buf)[2 * i1 + comp] = x;
    reinterpret_cast<double*>(buf)[2 * i2 + comp] = -x;
  }
};

struct ArithF {
  using V = float2;
  using R = float;
  using Sc = float;
  static __device__ __forceinline__ Sc make_sc(double s) { return (float)s; }
  static __device__ __forceinline__ Sc row_sc(const double*, const float* t32, int p) { return t32[p]; }
  static __device__ __forceinline__ V scale_sc(V a, Sc s) { return make_float2(a.x * s, a.y * s); }
  static __device__ __forceinline__ Sc neg_imag_sc(V a) { return -a.y; }
  // the scaled loads and read-outs of the FP32 time pass use the cheaper conversions
  static __device__ __forceinline__ double part_sc(V a, int comp, Sc s) { return f2d_fast((comp ? a.y : a.x) * s); }
  static __device__ __forceinline__ void put_sc(V* buf, int idx, int comp, double x, Sc s) {
    reinterpret_cast<float*>(buf)[2 * idx + comp] = d2f_fast(x) * s;
  }
  static __device__ __forceinline__ void put_sc2(V* buf, int i1, int i2, int comp, double x, Sc s) {
    const float v = d2f_bits(x) * s;
    reinterpret_cast<float*>(buf)[2 * i1 + comp] = v;
    reinterpret_cast<float*>(buf)[2 * i2 + comp] = v;
  }
  static __device__ __forceinline__ V add(V a, V b) { return make_float2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ V sub(V a, V b) { return make_float2(a.x - b.x, a.y - b.y); }
  static __device__ __forceinline__ V add_nr(V a, V b) { return add(a, b); }
  static __device__ __forceinline__ V sub_nr(V a, V b) { return sub(a, b); }
  static __device__ __forceinline__ V conj(V a) { return make_float2(a.x, -a.y); }
  static __device__ __forceinline__ V mul(V a, V b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
  }
  static __device__ __forceinline__ V mulc(V a, V b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
  }
  static __device__ __forceinline__ V mul_nr(V a, V b) { return mul(a, b); }
  static __device__ __forceinline__ V mulc_nr(V a, V b) { return mulc(a, b); }
  template <bool INV> static __device__ __forceinline__ V rot(V a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
  }
  static __device__ __forceinline__ V scale(V a, double s) {
    float f = (float)s;
    return make_float2(a.x * f, a.y * f);
  }
  static __device__ __forceinline__ V zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ V from(double re, double im) { return make_float2((float)re, (float)im); }
  static __device__ __forceinline__ V cst(double, double, float rh, float, float ih, float) {
    return make_float2(rh, ih);
  }
  static __device__ __forceinline__ double part(V a, int comp) { return f2d_bits(comp ? a.y : a.x); }
  static __device__ __forceinline__ void put(V* buf, int idx, int comp, double x) {
    reinterpret_cast<float*>(buf)[2 * idx + comp] = d2f_bits(x);
  }
  static __device__ __forceinline__ void put_pm(V* buf, int i1, int i2, int comp, double x) {
    const float f = d2f_bits(x);
    reinterpret_cast<float*>(buf)[2 * i1 + comp] = f;
    reinterpret_cast<float*>(buf)[2 * i2 + comp] = -f;
  }
};

// complex double-float packed as float4 {re.hi, re.lo, im.hi, im.lo}
struct ArithDF {
  using V = float4;
  using R = dfl;
  using Sc = dfl;
  static __device__ __forceinline__ Sc make_sc(double s) { return df_from(s); }
  static __device__ __forceinline__ Sc row_sc(const float2* tdf, int p) { const float2 v = tdf[p]; return {v.x, v.y}; }
  static __device__ __forceinline__ V scale_sc(V a, Sc s) {
    return pack(df_mul(dfl{a.x, a.y}, s), df_mul(dfl{a.z, a.w}, s));
  }
  static __device__ __forceinline__ Sc neg_imag_sc(V a) { return {-a.z, -a.w}; }
  static __device__ __forceinline__ double part_sc(V a, int comp, Sc s) {
    return df_to(df_mul(comp ? dfl{a.z, a.w} : dfl{a.x, a.y}, s));
  }
  static __device__ __forceinline__ void put_sc(V* buf, int idx, int comp, double x, Sc s) {
    dfl v = df_mul(df_from(x), s);
    reinterpret_cast<float2*>(buf)[2 * idx + comp] = make_float2(v.hi, v.lo);
  }
  // the same value into two slots, converted and scaled once
  static __device__ __forceinline__ void put_sc2(V* buf, int i1, int i2, int comp, double x, Sc s) {
    const dfl v = df_mul(df_from(x), s);
    reinterpret_cast<float2*>(buf)[2 * i1 + comp] = make_float2(v.hi, v.lo);
    reinterpret_cast<float2*>(buf)[2 * i2 + comp] = make_float2(v.hi, v.lo);
  }
  static __device__ __forceinline__ dfl re(V a) { return {a.x, a.y}; }
  static __device__ __forceinline__ dfl im(V a) { return {a.z, a.w}; }
  static __device__ __forceinline__ V pack(dfl r, dfl i) { return make_float4(r.hi, r.lo, i.hi, i.lo); }
  static __device__ __forceinline__ V add(V a, V b) { return pack(df_add(re(a), re(b)), df_add(im(a), im(b))); }
  static __device__ __forceinline__ V sub(V a, V b) { return pack(df_sub(re(a), re(b)), df_sub(im(a), im(b))); }
  // without the final renormalisation (intermediate sums of a butterfly)
  static __device__ __forceinline__ V add_nr(V a, V b) { return pack(df_add_nr(re(a), re(b)), df_add_nr(im(a), im(b))); }
  static __device__ __forceinline__ V sub_nr(V a, V b) { return pack(df_sub_nr(re(a), re(b)), df_sub_nr(im(a), im(b))); }
  static __device__ __forceinline__ V conj(V a) { return make_float4(a.x, a.y, -a.z, -a.w); }
  static __device__ __forceinline__ V mul(V a, V b) {
    return pack(df_dot2(re(a), re(b), df_neg(im(a)), im(b)), df_dot2(re(a), im(b), im(a), re(b)));
  }
  static __device__ __forceinline__ V mulc(V a, V b) {
    return pack(df_dot2(re(a), re(b), im(a), im(b)), df_dot2(im(a), re(b), df_neg(re(a)), im(b)));
  }
  // products that only feed the first (non-renormalising) level of a butterfly
  static __device__ __forceinline__ V mul_nr(V a, V b) {
    return pack(df_dot2_nr(re(a), re(b), df_neg(im(a)), im(b)), df_dot2_nr(re(a), im(b), im(a), re(b)));
  }
  static __device__ __forceinline__ V mulc_nr(V a, V b) {
    return pack(df_dot2_nr(re(a), re(b), im(a), im(b)), df_dot2_nr(im(a), re(b), df_neg(re(a)), im(b)));
  }
  template <bool INV> static __device__ __forceinline__ V rot(V a) {
    return INV ? make_float4(-a.z, -a.w, a.x, a.y) : make_float4(a.z, a.w, -a.x, -a.y);
  }
  static __device__ __forceinline__ V scale(V a, double s) {
    dfl f = df_from(s);
    return pack(df_mul(re(a), f), df_mul(im(a), f));
  }
  static __device__ __forceinline__ V zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ V cst(double, double, float rh, float rl, float ih, float il) {
    return make_float4(rh, rl, ih, il);
  }
  static __device__ __forceinline__ V from(double r, double i) { return pack(df_from(r), df_from(i)); }
  static __device__ __forceinline__ double part(V a, int comp) {
    return comp ? df_to(im(a)) : df_to(re(a));
  }
  static __device__ __forceinline__ void put(V* buf, int idx, int comp, double x) {
    dfl v = df_from(x);
    reinterpret_cast<float2*>(buf)[2 * idx + comp] = make_float2(v.hi, v.lo);
  }
  static __device__ __forceinline__ void put_pm(V* buf, int i1, int i2, int comp, double x) {
    dfl v = df_from(x);
    reinterpret_cast<float2*>(buf)[2 * i1 + comp] = make_float2(v.hi, v.lo);
    reinterpret_cast<float2*>(buf)[2 * i2 + comp] = make_float2(-v.hi, -v.lo);
  }
};

// ------------------------------------------------------------------------------------------
// Radix-16 butterfly.  With r = b + 4c and q = c' + 4d (b, c, c', d < 4),
//   X_q = sum_b w4^{b d} w16^{b c'} sum_c w4^{c c'} x_{b+4c},
// i.e. four length-4 DFTs over c, the constant twiddles w16^{b c'}, and four length-4 DFTs over
// b.  w16 = exp(-2 pi i / 16) (forward) or its conjugate (INV).

// cos(pi/8), sin(pi/8) and sqrt(1/2): FP64 values and FP32 leading + trailing parts
struct K16 {
  static constexpr double C = 0.92387953251128674, S = 0.38268343236508978,
                          Q = 0.70710678118654752;
  static constexpr float Ch = 0x1.d906bcp-1f, Cl = 0x1.e651a8p-26f;
  static constexpr float Sh = 0x1.87de2ap-2f, Sl = 0x1.abaa58p-28f;
  static constexpr float Qh = 0x1.6a09e6p-1f, Ql = 0x1.9fcef4p-27f;
};

// w16^E for the exponents E in {1, 2, 3, 6, 9} that the butterfly needs (E = 4 is a rotation)
template <class A, int E, bool INV>
__device__ __forceinline__ typename A::V w16() {
  constexpr float g = INV ? -1.f : 1.f;   // sign of -Im
  using K = K16;
  if constexpr (E == 1) return A::cst(K::C, -g * K::S, K::Ch, K::Cl, -g * K::Sh, -g * K::Sl);
  else if constexpr (E == 2) return A::cst(K::Q, -g * K::Q, K::Qh, K::Ql, -g * K::Qh, -g * K::Ql);
  else if constexpr (E == 3) return A::cst(K::S, -g * K::C, K::Sh, K::Sl, -g * K::Ch, -g * K::Cl);
  else if constexpr (E == 6) return A::cst(-K::Q, -g * K::Q, -K::Qh, -K::Ql, -g * K::Qh, -g * K::Ql);
  else return A::cst(-K::C, g * K::S, -K::Ch, -K::Cl, g * K::Sh, g * K::Sl);   // E == 9
}

// Double-float sums inside the FFT passes are not renormalised.  A pair (s, e) left by a two-sum
// still represents its value exactly; without the final fast two-sum the trailing part may grow
// to a few ulp of the leading one over the levels of a transform, and the FP32 rounding of the
// trailing-part sums then costs about 2^-24 of that, i.e. of order L_levels * 2^-48 of the
// operands' size, far inside the FP64-accurate bound.  Every product that leaves a transform
// (spectral products, scalings, the conversion back to FP64) takes unnormalised pairs.
constexpr bool kFftNoRenorm = true;

// NR: the second level is not renormalised either.  HALF: only X_0 and X_1 are formed (x2, x3
// are left unchanged), for a last pass whose upper outputs are not needed.
template <class A, bool INV, bool NR = kFftNoRenorm, bool HALF = false>
__device__ __forceinline__ void dft4(typename A::V& x0, typename A::V& x1, typename A::V& x2,
                                     typename A::V& x3) {
  using V = typename A::V;
  // the first level's sums are not renormalised: they only feed the second level
  const V t0 = A::add_nr(x0, x2), t1 = A::sub_nr(x0, x2), t2 = A::add_nr(x1, x3);
  const V t3 = A::template rot<INV>(A::sub_nr(x1, x3));
  if constexpr (NR) {
    x0 = A::add_nr(t0, t2);
    x1 = A::add_nr(t1, t3);
    if constexpr (!HALF) {
      x2 = A::sub_nr(t0, t2);
      x3 = A::sub_nr(t1, t3);
    }
  } else {
    x0 = A::add(t0, t2);
    x1 = A::add(t1, t3);
    if constexpr (!HALF) {
      x2 = A::sub(t0, t2);
      x3 = A::sub(t1, t3);
    }
  }
}

// in place; on return X_{c' + 4d} is in v[4c' + d] (HALF: only d < 2 is formed)
template <class A, bool INV, bool HALF = false>
__device__ __forceinline__ void dft16(typename A::V (&v)[16]) {
#pragma unroll
  for (int b = 0; b < 4; ++b) dft4<A, INV>(v[b], v[b + 4], v[b + 8], v[b + 12]);
  v[5] = A::mul_nr(v[5], w16<A, 1, INV>());
  v[6] = A::mul_nr(v[6], w16<A, 2, INV>());
  v[7] = A::mul_nr(v[7], w16<A, 3, INV>());
  v[9] = A::mul_nr(v[9], w16<A, 2, INV>());
  v[10] = A::template rot<INV>(v[10]);
  v[11] = A::mul_nr(v[11], w16<A, 6, INV>());
  v[13] = A::mul_nr(v[13], w16<A, 3, INV>());
  v[14] = A::mul_nr(v[14], w16<A, 6, INV>());
  v[15] = A::mul_nr(v[15], w16<A, 9, INV>());
#pragma unroll
  for (int c = 0; c < 4; ++c) dft4<A, INV, false, HALF>(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
}

// Radix-8 butterfly.  With r = b + 2c and q = c' + 4d (b, d < 2; c, c' < 4),
//   X_q = sum_b w2^{b d} w8^{b c'} sum_c w4^{c c'} x_{b+2c}:
// two length-4 DFTs over c, the twiddles w8^{c'} on the b = 1 half, four length-2 DFTs over b.
// In place; on return X_{c' + 4d} is in v[2c' + d] (HALF: only d = 0 is formed).
template <class A, bool INV, bool HALF = false>
__device__ __forceinline__ void dft8(typename A::V (&v)[8]) {
  dft4<A, INV, true>(v[0], v[2], v[4], v[6]);
  dft4<A, INV, true>(v[1], v[3], v[5], v[7]);
  v[3] = A::mul_nr(v[3], w16<A, 2, INV>());   // w8^1 = w16^2
  v[5] = A::template rot<INV>(v[5]);          // w8^2 = -i (forward)
  v[7] = A::mul_nr(v[7], w16<A, 6, INV>());   // w8^3 = w16^6
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const typename A::V a = v[2 * c], b = v[2 * c + 1];
    if constexpr (kFftNoRenorm) {
      v[2 * c] = A::add_nr(a, b);
      if constexpr (!HALF) v[2 * c + 1] = A::sub_nr(a, b);
    } else {
      v[2 * c] = A::add(a, b);
      if constexpr (!HALF) v[2 * c + 1] = A::sub(a, b);
    }
  }
}

// ------------------------------------------------------------------------------------------
// Shared-memory Stockham FFT (self-sorting, mixed radix).  With 16 points per thread (CAP = 16 NT)
// the passes are radix 2 when log2 L is odd, radix 4 when the remaining exponent is 2 mod 4, and
// radix 16 for the rest.  With at most 8 points per thread they are one or two radix-4 passes
// (exponent 2 or 1 mod 3) and radix 8 for the rest, with a radix-2 pass first only when the
// caller has applied it (skip_radix2) or L = 2.  Running the short passes first keeps the long
// ones at Ns >= 4, where their stores stay bank-conflict-free.
//
// buf holds NC = 2^log2NC independent complex columns of length L, element (p, c) at
// buf[p * NC + c] (or at buf[p * NC + (c ^ (p mod NC))] with SWZ).  tw holds
// w_L^k = exp(-2 pi i k / L), k < L, at tw[k << tw_shift] (a table of a 2^tw_shift times longer
// transform serves at that stride).  skip_radix2: the caller has already applied the first
// radix-2 pass (used when the upper half of the input is zero: the pass only duplicates).
// Forward: X_k = sum_j x_j w^{jk}; inverse (INV): conjugate twiddles, no 1/L scaling.  Every
// pass loads all of its butterfly inputs into registers, synchronises, then writes, so the
// transform runs in place.  CAP bounds NC * L; the block has NT threads.
//
// A pass of radix R with Ns outputs already combined: butterfly j (of L/R) reads x_{j + r L/R},
// multiplies input r by w_L^{r k L/(R Ns)} (k = j mod Ns), transforms, and writes output q at
// (j - k) R + k + q Ns.
//
// half_out: only the outputs X_k with k < L/2 are needed; a last pass of radix 8 or 16 then forms
// and stores only those (the rows L/2.. keep whatever they held).
template <class A, int NT, int CAP, bool INV, bool SWZ = false>
__device__ __forceinline__ void fft_columns(typename A::V* buf, int L, int log2L, int log2NC,
                            const typename A::V* __restrict__ tw, bool skip_radix2 = false,
                            int tw_shift = 0, bool half_out = false) {
  using V = typename A::V;
  constexpr int IPT2 = (CAP / 2 + NT - 1) / NT;
  constexpr int IPT4 = (CAP / 4 + NT - 1) / NT;
  constexpr int IPT16 = (CAP / 16 + NT - 1) / NT;
  const int tid = threadIdx.x;
  const int NC = 1 << log2NC, cmask = NC - 1;
  auto at = [&](int p, int c) { return (p << log2NC) + (SWZ ? (c ^ (p & cmask)) : c); };
  constexpr bool R8 = (CAP / NT) <= 8;   // radix-8 plan (at most 8 points per thread)
  int log2Ns = 0;
  // radix 2 first when log2 L is odd; the radix-8 plan needs it only when the caller has applied
  // it (skip_radix2) or for L = 2, and otherwise absorbs the odd level into its radix-4/8 passes
  if ((log2L & 1) && (!R8 || skip_radix2 || log2L == 1)) {
    if (!skip_radix2) {
      const int half = L >> 1;
      const int total = half << log2NC;
      V v[IPT2][2];
#pragma unroll
      for (int s = 0; s < IPT2; ++s) {
        const int it = tid + s * NT;
        if (it < total) {
          const int c = it & cmask, j = it >> log2NC;
          v[s][0] = buf[at(j, c)];
          v[s][1] = buf[at(j + half, c)];
        }
      }
      __syncthreads();
#pragma unroll
      for (int s = 0; s < IPT2; ++s) {
        const int it = tid + s * NT;
        if (it < total) {
          const int c = it & cmask, j = it >> log2NC;
          buf[at(2 * j, c)] = A::add_nr(v[s][0], v[s][1]);
          buf[at(2 * j + 1, c)] = A::sub_nr(v[s][0], v[s][1]);
        }
      }
      __syncthreads();
    }
    log2Ns = 1;
  }
  const int rem = log2L - log2Ns;
  const int n4 = R8 ? (rem % 3 == 2 ? 1 : (rem % 3 == 1 ? 2 : 0)) : ((rem & 2) ? 1 : 0);
  for (int i4 = 0; i4 < n4; ++i4) {
    const int Ns = 1 << log2Ns;
    const int quarter = L >> 2;
    const int total = quarter << log2NC;
    const int tstep_log = log2L - 2 - log2Ns;
    V v[IPT4][4];
#pragma unroll
    for (int s = 0; s < IPT4; ++s) {
      const int it = tid + s * NT;
      if (it < total) {
        const int c = it & cmask, j = it >> log2NC;
#pragma unroll
        for (int r = 0; r < 4; ++r) v[s][r] = buf[at(j + r * quarter, c)];
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < IPT4; ++s) {
      const int it = tid + s * NT;
      if (it < total) {
        const int c = it & cmask, j = it >> log2NC;
        const int k = j & (Ns - 1);
        if (k != 0) {
          const int e = k << (tstep_log + tw_shift);
#pragma unroll
          for (int r = 1; r < 4; ++r) {
            const V w = tw[r * e];
            v[s][r] = INV ? A::mulc_nr(v[s][r], w) : A::mul_nr(v[s][r], w);
          }
        }
        dft4<A, INV>(v[s][0], v[s][1], v[s][2], v[s][3]);
        const int o = (j - k) * 4 + k;
#pragma unroll
        for (int q = 0; q < 4; ++q) buf[at(o + q * Ns, c)] = v[s][q];
      }
    }
    __syncthreads();
    log2Ns += 2;
  }
  if constexpr (R8) {
    constexpr int IPT8 = (CAP / 8 + NT - 1) / NT;
    const int eighth = L >> 3;
    const int total8 = eighth << log2NC;
    for (; log2Ns < log2L; log2Ns += 3) {
      const int Ns = 1 << log2Ns;
      const int tstep_log = log2L - 3 - log2Ns;
      V v[IPT8][8];
#pragma unroll
      for (int s = 0; s < IPT8; ++s) {
        const int it = tid + s * NT;
        if (it < total8) {
          const int c = it & cmask, j = it >> log2NC;
#pragma unroll
          for (int r = 0; r < 8; ++r) v[s][r] = buf[at(j + r * eighth, c)];
        }
      }
      __syncthreads();
#pragma unroll
      for (int s = 0; s < IPT8; ++s) {
        const int it = tid + s * NT;
        if (it < total8) {
          const int c = it & cmask, j = it >> log2NC;
          const int k = j & (Ns - 1);
          if (k != 0) {
            const int e = k << (tstep_log + tw_shift);
#pragma unroll
            for (int r = 1; r < 8; ++r) {
              const V w = tw[r * e];
              v[s][r] = INV ? A::mulc_nr(v[s][r], w) : A::mul_nr(v[s][r], w);
            }
          }
          const int o = (j - k) * 8 + k;
          if (half_out && log2Ns + 3 == log2L) {
            // last pass: outputs q < 4 land in rows < L/2
            dft8<A, INV, true>(v[s]);
#pragma unroll
            for (int q = 0; q < 4; ++q) buf[at(o + q * Ns, c)] = v[s][2 * q];
          } else {
            dft8<A, INV>(v[s]);
#pragma unroll
            for (int q = 0; q < 8; ++q) buf[at(o + q * Ns, c)] = v[s][2 * (q & 3) + (q >> 2)];
          }
        }
      }
      __syncthreads();
    }
    return;
  }
  const int sixteenth = L >> 4;
  const int total16 = sixteenth << log2NC;
  for (; log2Ns < log2L; log2Ns += 4) {
    const int Ns = 1 << log2Ns;
    const int tstep_log = log2L - 4 - log2Ns;
    V v[IPT16][16];
#pragma unroll
    for (int s = 0; s < IPT16; ++s) {
      const int it = tid + s * NT;
      if (it < total16) {
        const int c = it & cmask, j = it >> log2NC;
#pragma unroll
        for (int r = 0; r < 16; ++r) v[s][r] = buf[at(j + r * sixteenth, c)];
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < IPT16; ++s) {
      const int it = tid + s * NT;
      if (it < total16) {
        const int c = it & cmask, j = it >> log2NC;
        const int k = j & (Ns - 1);
        if (k != 0) {
          const int e = k << (tstep_log + tw_shift);
#pragma unroll
          for (int r = 1; r < 16; ++r) {
            const V w = tw[r * e];
            v[s][r] = INV ? A::mulc_nr(v[s][r], w) : A::mul_nr(v[s][r], w);
          }
        }
        const int o = (j - k) * 16 + k;
        if (half_out && log2Ns + 4 == log2L) {
          // last pass: outputs q < 8 land in rows < L/2
          dft16<A, INV, true>(v[s]);
#pragma unroll
          for (int q = 0; q < 8; ++q) buf[at(o + q * Ns, c)] = v[s][4 * (q & 3) + (q >> 2)];
        } else {
          dft16<A, INV>(v[s]);
#pragma unroll
          for (int q = 0; q < 16; ++q) buf[at(o + q * Ns, c)] = v[s][4 * (q & 3) + (q >> 2)];
        }
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------
// block-wide sum of one double per thread; result valid in thread 0.  scratch: >= 32 doubles.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* scratch) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    r = (lane < NT / 32) ? scratch[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;
}

}  // namespace bltt
