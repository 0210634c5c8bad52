// Double-float arithmetic: every real is an unevaluated sum hi + lo of two fp32 values
// (~48-bit significand), with Knuth's two-sum for additions and the FMA-based exact product
// for multiplications (Dekker's product, FMA form). The B300 issues fp64 at 1/64 of its
// fp32 rate, so fp64-accurate kernels whose inner loops are multiply-adds (the complex128
// transforms, the fp64 pair sum) compute in these pairs; their global arrays stay
// complex128.
#pragma once
#include "dev.cuh"

namespace tmat {

struct DF {};
struct dfc {
  float rh, rl, ih, il;
};
template <> struct cplx<DF> { using t = dfc; };
// global element type of a transform's compute type (double-float reads/writes complex128)
template <typename R> struct gtype { using t = C<R>; };
template <> struct gtype<DF> { using t = double2; };
template <typename R> using G = typename gtype<R>::t;

__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void df_norm(float& h, float& l) {  // quick two-sum, |h| >= |l|
  const float s = h + l;
  l = l - (s - h);
  h = s;
}
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& h, float& l) {
  float s, e;
  df_two_sum(ah, bh, s, e);
  e += al + bl;
  h = s;
  l = e;
  df_norm(h, l);
}
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& h, float& l) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, fmaf(al, bh, e));
  h = p;
  l = e;
  df_norm(h, l);
}
__device__ __forceinline__ dfc cadd(dfc a, dfc b) {
  dfc z;
  df_add(a.rh, a.rl, b.rh, b.rl, z.rh, z.rl);
  df_add(a.ih, a.il, b.ih, b.il, z.ih, z.il);
  return z;
}
__device__ __forceinline__ dfc csub(dfc a, dfc b) {
  dfc z;
  df_add(a.rh, a.rl, -b.rh, -b.rl, z.rh, z.rl);
  df_add(a.ih, a.il, -b.ih, -b.il, z.ih, z.il);
  return z;
}
__device__ __forceinline__ dfc cmul(dfc a, dfc b) {
  float p1h, p1l, p2h, p2l, p3h, p3l, p4h, p4l;
  df_mul(a.rh, a.rl, b.rh, b.rl, p1h, p1l);
  df_mul(a.ih, a.il, b.ih, b.il, p2h, p2l);
  df_mul(a.rh, a.rl, b.ih, b.il, p3h, p3l);
  df_mul(a.ih, a.il, b.rh, b.rl, p4h, p4l);
  dfc z;
  df_add(p1h, p1l, -p2h, -p2l, z.rh, z.rl);
  df_add(p3h, p3l, p4h, p4l, z.ih, z.il);
  return z;
}

template <typename R> __device__ __forceinline__ C<R> czero() { return mk<R>((R)0, (R)0); }
template <> __device__ __forceinline__ dfc czero<DF>() { return dfc{0.f, 0.f, 0.f, 0.f}; }
__device__ __forceinline__ void df_split(double v, float& h, float& l) {
  h = (float)v;
  l = (float)(v - (double)h);
}
template <typename R> __device__ __forceinline__ C<R> cfrom64(double re, double im) { return mk<R>((R)re, (R)im); }
template <> __device__ __forceinline__ dfc cfrom64<DF>(double re, double im) {
  dfc z;
  df_split(re, z.rh, z.rl);
  df_split(im, z.ih, z.il);
  return z;
}
template <typename R> __device__ __forceinline__ C<R> gload(G<R> v) { return v; }
template <> __device__ __forceinline__ dfc gload<DF>(double2 v) { return cfrom64<DF>(v.x, v.y); }
template <typename R> __device__ __forceinline__ G<R> gstore(C<R> v) { return v; }
template <> __device__ __forceinline__ double2 gstore<DF>(dfc v) {
  return make_double2((double)v.rh + (double)v.rl, (double)v.ih + (double)v.il);
}
// times -i (dir < 0) or +i (dir > 0): exact
template <typename R> __device__ __forceinline__ C<R> crot(C<R> t, int dir) {
  return dir < 0 ? mk<R>(t.y, -t.x) : mk<R>(-t.y, t.x);
}
template <> __device__ __forceinline__ dfc crot<DF>(dfc t, int dir) {
  return dir < 0 ? dfc{t.ih, t.il, -t.rh, -t.rl} : dfc{-t.ih, -t.il, t.rh, t.rl};
}

__device__ __forceinline__ dfc cconj(dfc a) {
  a.ih = -a.ih;
  a.il = -a.il;
  return a;
}
// (h, l) += a b - c d
__device__ __forceinline__ void df_fma2(float& h, float& l, float ah, float al, float bh, float bl, float ch, float cl,
                                        float dh, float dl) {
  const float p = ah * bh;
  float pe = fmaf(ah, bh, -p);
  pe = fmaf(ah, bl, fmaf(al, bh, pe));
  const float m = ch * dh;
  float me = fmaf(ch, dh, -m);
  me = fmaf(ch, dl, fmaf(cl, dh, me));
  float s1, e1, s2, e2;
  df_two_sum(h, p, s1, e1);
  df_two_sum(s1, -m, s2, e2);
  l = l + e1 + e2 + pe - me;
  h = s2;
  df_norm(h, l);
}
// acc += a b
__device__ __forceinline__ void cfma(dfc& acc, dfc a, dfc b) {
  df_fma2(acc.rh, acc.rl, a.rh, a.rl, b.rh, b.rl, a.ih, a.il, b.ih, b.il);
  df_fma2(acc.ih, acc.il, a.rh, a.rl, b.ih, b.il, -a.ih, -a.il, b.rh, b.rl);
}
// a times the real double-float (vh, vl)
__device__ __forceinline__ dfc cscale_df(dfc a, float vh, float vl) {
  dfc z;
  df_mul(a.rh, a.rl, vh, vl, z.rh, z.rl);
  df_mul(a.ih, a.il, vh, vl, z.ih, z.il);
  return z;
}

}  // namespace tmat
