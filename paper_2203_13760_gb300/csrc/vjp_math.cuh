// Reverse-mode (vector-Jacobian) counterparts of the point-wise numerics in
// jf_math.cuh, written by hand.  Each function recomputes the forward values
// it needs and adds input cotangents for a given output cotangent.  Branches
// (min / max of the signal speeds, the HLLC side, the safe-reconstruction
// fallback) follow the branch the forward values take.
//
// References (arXiv 2203.13760): Section 3.3 (WENO5-JS face states, HLLC flux
// with Einfeldt speeds), Section 2 / 3.4 (dissipative fluxes), Section 7.2
// (gradients propagated back through the solver).
#pragma once
#include "jf_math.cuh"

namespace jf {

// weno5 (left-biased value from v0..v4 = v[i-2..i+2]): vb[k] += yb * dy/dv_k.
template <typename T>
JF_HD void weno5_vjp(T v0, T v1, T v2, T v3, T v4, T eps, T yb, T vb[5]) {
  const T sixth = T(1) / T(6);
  const T q0 = (T(2) * v0 - T(7) * v1 + T(11) * v2) * sixth;
  const T q1 = (-v1 + T(5) * v2 + T(2) * v3) * sixth;
  const T q2 = (T(2) * v2 + T(5) * v3 - v4) * sixth;
  const T c13 = T(13) / T(12);
  const T d0 = v0 - T(2) * v1 + v2, e0 = v0 - T(4) * v1 + T(3) * v2;
  const T d1 = v1 - T(2) * v2 + v3, e1 = v1 - v3;
  const T d2 = v2 - T(2) * v3 + v4, e2 = T(3) * v2 - T(4) * v3 + v4;
  const T t0 = eps + c13 * d0 * d0 + T(0.25) * e0 * e0;
  const T t1 = eps + c13 * d1 * d1 + T(0.25) * e1 * e1;
  const T t2 = eps + c13 * d2 * d2 + T(0.25) * e2 * e2;
  // every division through a reciprocal (trcp: approximate in FP32 device code)
  const T r0 = trcp(t0), r1 = trcp(t1), r2 = trcp(t2);
  const T a0 = T(0.1) * r0 * r0, a1 = T(0.6) * r1 * r1, a2 = T(0.3) * r2 * r2;
  const T inv = trcp(a0 + a1 + a2);
  const T y = (a0 * q0 + a1 * q1 + a2 * q2) * inv;
  const T s = yb * inv;
  const T qb0 = s * a0, qb1 = s * a1, qb2 = s * a2;
  // d alpha_k / d t_k = -2 alpha_k / t_k;  beta_k enters t_k with slope 1
  const T tb0 = -T(2) * s * (q0 - y) * a0 * r0;
  const T tb1 = -T(2) * s * (q1 - y) * a1 * r1;
  const T tb2 = -T(2) * s * (q2 - y) * a2 * r2;
  const T db0 = T(2) * c13 * d0 * tb0, eb0 = T(0.5) * e0 * tb0;
  const T db1 = T(2) * c13 * d1 * tb1, eb1 = T(0.5) * e1 * tb1;
  const T db2 = T(2) * c13 * d2 * tb2, eb2 = T(0.5) * e2 * tb2;
  vb[0] += db0 + eb0 + T(2) * sixth * qb0;
  vb[1] += -T(2) * db0 - T(4) * eb0 + db1 + eb1 - T(7) * sixth * qb0 - sixth * qb1;
  vb[2] += db0 + T(3) * eb0 - T(2) * db1 + db2 + T(3) * eb2 + T(11) * sixth * qb0 + T(5) * sixth * qb1 +
           T(2) * sixth * qb2;
  vb[3] += db1 - eb1 - T(2) * db2 - T(4) * eb2 + T(2) * sixth * qb1 + T(5) * sixth * qb2;
  vb[4] += db2 + eb2 - sixth * qb2;
}

#ifdef __CUDACC__
// weno5_vjp for two stencils at once in packed FP32x2 arithmetic (lane x:
// v0..v4 = v[i-2..i+2] -> v^-, lane y: the mirrored stencil -> v^+, as in
// weno5_pair): vb[k] = yb * dy/dv_k per lane (assigned, not added).  The
// same formulas as weno5_vjp, grouped into fused multiply-adds.
__device__ __forceinline__ void weno5_vjp_pair(float2 v0, float2 v1, float2 v2, float2 v3, float2 v4, float eps,
                                               float2 yb, float2 vb[5]) {
  auto c = [](float x) { return make_float2(x, x); };
  auto rcp2 = [](float2 x) { return make_float2(__fdividef(1.0f, x.x), __fdividef(1.0f, x.y)); };
  const float2 q0 = __ffma2_rn(c(11.0f / 6.0f), v2, __ffma2_rn(c(-7.0f / 6.0f), v1, __fmul2_rn(c(2.0f / 6.0f), v0)));
  const float2 q1 = __ffma2_rn(c(2.0f / 6.0f), v3, __ffma2_rn(c(5.0f / 6.0f), v2, __fmul2_rn(c(-1.0f / 6.0f), v1)));
  const float2 q2 = __ffma2_rn(c(-1.0f / 6.0f), v4, __ffma2_rn(c(5.0f / 6.0f), v3, __fmul2_rn(c(2.0f / 6.0f), v2)));
  const float2 d0 = __ffma2_rn(c(-2.0f), v1, __fadd2_rn(v0, v2));
  const float2 e0 = __ffma2_rn(c(3.0f), v2, __ffma2_rn(c(-4.0f), v1, v0));
  const float2 d1 = __ffma2_rn(c(-2.0f), v2, __fadd2_rn(v1, v3));
  const float2 e1 = __ffma2_rn(c(-1.0f), v3, v1);
  const float2 d2 = __ffma2_rn(c(-2.0f), v3, __fadd2_rn(v2, v4));
  const float2 e2 = __ffma2_rn(c(3.0f), v2, __ffma2_rn(c(-4.0f), v3, v4));
  const float2 k13 = c(13.0f / 12.0f), kq = c(0.25f), ke = c(eps);
  const float2 t0 = __ffma2_rn(__fmul2_rn(k13, d0), d0, __ffma2_rn(__fmul2_rn(kq, e0), e0, ke));
  const float2 t1 = __ffma2_rn(__fmul2_rn(k13, d1), d1, __ffma2_rn(__fmul2_rn(kq, e1), e1, ke));
  const float2 t2 = __ffma2_rn(__fmul2_rn(k13, d2), d2, __ffma2_rn(__fmul2_rn(kq, e2), e2, ke));
  const float2 r0 = rcp2(t0), r1 = rcp2(t1), r2 = rcp2(t2);
  const float2 a0 = __fmul2_rn(__fmul2_rn(c(0.1f), r0), r0);
  const float2 a1 = __fmul2_rn(__fmul2_rn(c(0.6f), r1), r1);
  const float2 a2 = __fmul2_rn(__fmul2_rn(c(0.3f), r2), r2);
  const float2 inv = rcp2(__fadd2_rn(__fadd2_rn(a0, a1), a2));
  const float2 y = __fmul2_rn(__ffma2_rn(a2, q2, __ffma2_rn(a1, q1, __fmul2_rn(a0, q0))), inv);
  const float2 s = __fmul2_rn(yb, inv);
  const float2 qb0 = __fmul2_rn(s, a0), qb1 = __fmul2_rn(s, a1), qb2 = __fmul2_rn(s, a2);
  // d alpha_k / d t_k = -2 alpha_k / t_k: tb_k = -2 qb_k (q_k - y) r_k
  const float2 m1 = c(-1.0f), m2 = c(-2.0f);
  const float2 tb0 = __fmul2_rn(__fmul2_rn(m2, qb0), __fmul2_rn(__ffma2_rn(m1, y, q0), r0));
  const float2 tb1 = __fmul2_rn(__fmul2_rn(m2, qb1), __fmul2_rn(__ffma2_rn(m1, y, q1), r1));
  const float2 tb2 = __fmul2_rn(__fmul2_rn(m2, qb2), __fmul2_rn(__ffma2_rn(m1, y, q2), r2));
  const float2 k26 = c(13.0f / 6.0f), kh = c(0.5f);
  const float2 db0 = __fmul2_rn(__fmul2_rn(k26, d0), tb0), eb0 = __fmul2_rn(__fmul2_rn(kh, e0), tb0);
  const float2 db1 = __fmul2_rn(__fmul2_rn(k26, d1), tb1), eb1 = __fmul2_rn(__fmul2_rn(kh, e1), tb1);
  const float2 db2 = __fmul2_rn(__fmul2_rn(k26, d2), tb2), eb2 = __fmul2_rn(__fmul2_rn(kh, e2), tb2);
  vb[0] = __ffma2_rn(c(2.0f / 6.0f), qb0, __fadd2_rn(db0, eb0));
  vb[1] = __ffma2_rn(c(-1.0f / 6.0f), qb1,
                     __ffma2_rn(c(-7.0f / 6.0f), qb0,
                                __fadd2_rn(__fadd2_rn(db1, eb1), __ffma2_rn(c(-4.0f), eb0, __fmul2_rn(m2, db0)))));
  vb[2] = __ffma2_rn(c(2.0f / 6.0f), qb2,
                     __ffma2_rn(c(5.0f / 6.0f), qb1,
                                __ffma2_rn(c(11.0f / 6.0f), qb0,
                                           __ffma2_rn(c(3.0f), eb2,
                                                      __fadd2_rn(__ffma2_rn(m2, db1, db2),
                                                                 __ffma2_rn(c(3.0f), eb0, db0))))));
  vb[3] = __ffma2_rn(c(5.0f / 6.0f), qb2,
                     __ffma2_rn(c(2.0f / 6.0f), qb1,
                                __ffma2_rn(c(-4.0f), eb2, __ffma2_rn(m2, db2, __ffma2_rn(m1, eb1, db1)))));
  vb[4] = __ffma2_rn(c(-1.0f / 6.0f), qb2, __fadd2_rn(db2, eb2));
}
#endif

// hllc<T, D>: given Fb = dLoss/dF, set WLb, WRb = dLoss/dWL, dLoss/dWR.
template <typename T, int D>
JF_HD void hllc_vjp(const T WL[5], const T WR[5], const Gas<T>& g, const T Fb[5], T WLb[5],
                                         T WRb[5]) {
  // ---- forward (as in hllc) ----
  const T rL = WL[0], rR = WR[0], pL = WL[4], pR = WR[4];
  const T unL = WL[1 + D], unR = WR[1 + D];
  const T q2L = WL[1] * WL[1] + WL[2] * WL[2] + WL[3] * WL[3];
  const T q2R = WR[1] * WR[1] + WR[2] * WR[2] + WR[3] * WR[3];
  const T EL = pL * g.inv_gm1 + T(0.5) * rL * q2L;
  const T ER = pR * g.inv_gm1 + T(0.5) * rR * q2R;
  const T irL = trcp(rL), irR = trcp(rR);
  const T cL = tsqrt(g.gamma * pL * irL);
  const T cR = tsqrt(g.gamma * pR * irR);
  const T sL = tsqrt(rL), sR = tsqrt(rR);
  const T is = trcp(sL + sR);
  const T HL = (EL + pL) * irL, HR = (ER + pR) * irR;
  T ut[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) ut[m] = (sL * WL[1 + m] + sR * WR[1 + m]) * is;
  const T Ht = (sL * HL + sR * HR) * is;
  const T ct = tsqrt(g.gm1 * (Ht - T(0.5) * (ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2])));
  const T unt = ut[D];
  const T aL = unL - cL, bL = unt - ct;
  const bool selL = bL < aL;  // S_L = min(aL, bL) takes bL
  const T SL = selL ? bL : aL;
  const T aR = unR + cR, bR = unt + ct;
  const bool selR = aR < bR;  // S_R = max(aR, bR) takes bR
  const T SR = selR ? bR : aR;
  const T mL = rL * (SL - unL), mR = rR * (SR - unR);
  const T den = mL - mR, iden = trcp(den);
  const T Ss = (pR - pL + mL * unL - mR * unR) * iden;
  const bool left = (SL >= T(0)) || (Ss >= T(0));
  const bool star = left ? !(SL >= T(0)) : (SR > T(0));

  // ---- reverse ----
  T rLb = 0, rRb = 0, pLb = 0, pRb = 0, ELb = 0, ERb = 0, SLb = 0, SRb = 0, mLb = 0, mRb = 0, Ssb = 0;
  T wLb[3] = {0, 0, 0}, wRb[3] = {0, 0, 0};
  const T r = left ? rL : rR, p = left ? pL : pR, E = left ? EL : ER;
  const T w[3] = {left ? WL[1] : WR[1], left ? WL[2] : WR[2], left ? WL[3] : WR[3]};
  const T un = w[D];
  const T S = left ? SL : SR, m = left ? mL : mR;
  T rb = 0, pb = 0, Eb = 0, Sb = 0, mb = 0;
  T wb[3] = {0, 0, 0};
  if (star) {
    // F = F_K + S (U*_K - U_K)
    const T ir = left ? irL : irR, im = trcp(m);
    const T dS = S - Ss, idS = trcp(dS);
    const T fac = m * idS;
    const T X = E * ir + (Ss - un) * (Ss + p * im);
    T Us[5] = {fac, fac * w[0], fac * w[1], fac * w[2], fac * X};
    Us[1 + D] = fac * Ss;
    const T Uk[5] = {r, r * w[0], r * w[1], r * w[2], E};
#pragma unroll
    for (int q = 0; q < 5; ++q) Sb += Fb[q] * (Us[q] - Uk[q]);
    // U_K = [r, r w, E]
    rb -= S * Fb[0];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      rb -= S * Fb[1 + a] * w[a];
      wb[a] -= S * Fb[1 + a] * r;
    }
    Eb -= S * Fb[4];
    // U*_K = fac [1, w (S* in the normal slot), X]
    T facb = S * Fb[0] + S * Fb[4] * X;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a == D) {
        facb += S * Fb[1 + a] * Ss;
        Ssb += S * Fb[1 + a] * fac;
      } else {
        facb += S * Fb[1 + a] * w[a];
        wb[a] += S * Fb[1 + a] * fac;
      }
    }
    const T Xb = S * Fb[4] * fac;
    // X = E / r + (S* - un)(S* + p / m)
    const T A = Ss - un, B = Ss + p * im;
    Eb += Xb * ir;
    rb -= Xb * E * ir * ir;
    const T Ab = Xb * B, Bb = Xb * A;
    Ssb += Ab + Bb;
    wb[D] -= Ab;
    pb += Bb * im;
    mb -= Bb * p * im * im;
    // fac = m / (S - S*)
    mb += facb * idS;
    Sb -= facb * fac * idS;
    Ssb += facb * fac * idS;
  }
  // physical flux F_K = [r un, r un w, un (E + p)] + p e_normal (cotangent Fb)
  {
    const T mass = r * un;
    T massb = Fb[0];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      massb += Fb[1 + a] * w[a];
      wb[a] += Fb[1 + a] * mass;
    }
    pb += Fb[1 + D];
    wb[D] += Fb[4] * (E + p);
    Eb += Fb[4] * un;
    pb += Fb[4] * un;
    rb += massb * un;
    wb[D] += massb * r;
  }
  if (left) {
    rLb += rb; pLb += pb; ELb += Eb; SLb += Sb; mLb += mb;
#pragma unroll
    for (int a = 0; a < 3; ++a) wLb[a] += wb[a];
  } else {
    rRb += rb; pRb += pb; ERb += Eb; SRb += Sb; mRb += mb;
#pragma unroll
    for (int a = 0; a < 3; ++a) wRb[a] += wb[a];
  }
  if (star) {
    // S* = (pR - pL + mL unL - mR unR) / (mL - mR)
    const T numb = Ssb * iden, denb = -Ssb * Ss * iden;
    pRb += numb;
    pLb -= numb;
    mLb += numb * unL + denb;
    wLb[D] += numb * mL;
    mRb += -numb * unR - denb;
    wRb[D] -= numb * mR;
    // m_K = r_K (S_K - un_K)
    rLb += mLb * (SL - unL);
    SLb += mLb * rL;
    wLb[D] -= mLb * rL;
    rRb += mRb * (SR - unR);
    SRb += mRb * rR;
    wRb[D] -= mRb * rR;
    // Einfeldt speeds
    T untb = 0, ctb = 0, cLb = 0, cRb = 0;
    if (selL) { untb += SLb; ctb -= SLb; } else { wLb[D] += SLb; cLb -= SLb; }
    if (selR) { untb += SRb; ctb += SRb; } else { wRb[D] += SRb; cRb += SRb; }
    // c~ = sqrt(Z), Z = (gamma - 1)(H~ - |u~|^2 / 2)
    const T Zb = ctb * T(0.5) * trcp(ct);
    const T Htb = Zb * g.gm1;
    T utb[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) utb[a] = -Zb * g.gm1 * ut[a];
    utb[D] += untb;
    // H~ = (sL HL + sR HR) is ;  u~ = (sL wL + sR wR) is ;  is = 1 / (sL + sR)
    T sLb = Htb * HL * is, sRb = Htb * HR * is;
    const T HLb = Htb * sL * is, HRb = Htb * sR * is;
    T isb = Htb * (sL * HL + sR * HR);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      sLb += utb[a] * WL[1 + a] * is;
      sRb += utb[a] * WR[1 + a] * is;
      wLb[a] += utb[a] * sL * is;
      wRb[a] += utb[a] * sR * is;
      isb += utb[a] * (sL * WL[1 + a] + sR * WR[1 + a]);
    }
    const T ssb = -isb * is * is;
    sLb += ssb;
    sRb += ssb;
    // H_K = (E_K + p_K) / r_K
    ELb += HLb * irL;
    pLb += HLb * irL;
    rLb -= HLb * HL * irL;
    ERb += HRb * irR;
    pRb += HRb * irR;
    rRb -= HRb * HR * irR;
    // s_K = sqrt(r_K): d s / d r = 1 / (2 s) = s / (2 r)
    rLb += sLb * T(0.5) * sL * irL;
    rRb += sRb * T(0.5) * sR * irR;
    // c_K = sqrt(gamma p_K / r_K)
    const T zLb = cLb * T(0.5) * trcp(cL), zRb = cRb * T(0.5) * trcp(cR);
    pLb += zLb * g.gamma * irL;
    rLb -= zLb * g.gamma * pL * irL * irL;
    pRb += zRb * g.gamma * irR;
    rRb -= zRb * g.gamma * pR * irR * irR;
  }
  // E_K = p_K / (gamma - 1) + r_K |w_K|^2 / 2
  pLb += ELb * g.inv_gm1;
  rLb += ELb * T(0.5) * q2L;
  pRb += ERb * g.inv_gm1;
  rRb += ERb * T(0.5) * q2R;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    wLb[a] += ELb * rL * WL[1 + a];
    wRb[a] += ERb * rR * WR[1 + a];
  }
  WLb[0] = rLb; WLb[1] = wLb[0]; WLb[2] = wLb[1]; WLb[3] = wLb[2]; WLb[4] = pLb;
  WRb[0] = rRb; WRb[1] = wRb[0]; WRb[2] = wRb[1]; WRb[3] = wRb[2]; WRb[4] = pRb;
}

}  // namespace jf
