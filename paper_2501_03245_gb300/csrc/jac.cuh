// Jacobian-coordinate point arithmetic (x = X/Z^2, y = Y/Z^3; Section 2.1.2,
// Table 1), used where a phase is a long dependent chain per thread with too
// little parallelism to amortise a batch inversion: the MSM bucket reduction and
// window combination.  Z = 0 encodes O.  Coordinates are in Montgomery form.
// The group operations come in two forms: out of line (jac_dbl, jac_add: one
// copy per curve keeps code size and compile time small where many call sites
// use them) and inline (jac_dbl_inl, jac_add_inl: register-resident operands for
// the one long chain of the window combination).
#pragma once
#include "ec.cuh"

namespace ecc {

template <class F>
struct Jac {
  uint32_t X[F::N], Y[F::N], Z[F::N];
};

template <class C>
ECC_DEV void jac_set_inf(Jac<typename C::Fp>& P) {
  using F = typename C::Fp;
  fe_set_one<F>(P.X);
  fe_set_one<F>(P.Y);
  fe_set_zero<F>(P.Z);
}

template <class C>
ECC_DEV bool jac_is_inf(const Jac<typename C::Fp>& P) {
  return fe_is_zero<typename C::Fp>(P.Z);
}

// affine (x, y) with (0, 0) = O -> Jacobian
template <class C>
ECC_DEV void jac_from_affine(Jac<typename C::Fp>& P, const uint32_t* x, const uint32_t* y) {
  using F = typename C::Fp;
  if (pt_is_inf<F>(x, y)) {
    jac_set_inf<C>(P);
  } else {
    fe_copy<F>(P.X, x);
    fe_copy<F>(P.Y, y);
    fe_set_one<F>(P.Z);
  }
}

// 2P: S = 2((X + Y^2)^2 - X^2 - Y^4), M = 3 X^2 + a Z^4,
// X3 = M^2 - 2S, Y3 = M (S - X3) - 8 Y^4, Z3 = (Y + Z)^2 - Y^2 - Z^2.
template <class C>
ECC_DEV void jac_dbl_inl(Jac<typename C::Fp>& R, const Jac<typename C::Fp>& P) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  if (jac_is_inf<C>(P) || fe_is_zero<F>(P.Y)) {
    jac_set_inf<C>(R);
    return;
  }
  uint32_t XX[N], YY[N], YYYY[N], ZZ[N], S[N], M[N], t[N];
  mont_sqr<F>(XX, P.X);
  mont_sqr<F>(YY, P.Y);
  mont_sqr<F>(YYYY, YY);
  mont_sqr<F>(ZZ, P.Z);
  fe_add<F>(t, P.X, YY);
  mont_sqr<F>(t, t);
  fe_sub<F>(t, t, XX);
  fe_sub<F>(t, t, YYYY);
  fe_add<F>(S, t, t);
  fe_add<F>(M, XX, XX);
  fe_add<F>(M, M, XX);
  if (!C::A_ZERO) {
    uint32_t a[N];
    curve_a<C>(a);
    mont_sqr<F>(t, ZZ);
    mont_mul<F>(t, t, a);
    fe_add<F>(M, M, t);
  }
  uint32_t X3[N], Y3[N], Z3[N];
  fe_add<F>(Z3, P.Y, P.Z);
  mont_sqr<F>(Z3, Z3);
  fe_sub<F>(Z3, Z3, YY);
  fe_sub<F>(Z3, Z3, ZZ);
  mont_sqr<F>(X3, M);
  fe_sub<F>(X3, X3, S);
  fe_sub<F>(X3, X3, S);
  fe_sub<F>(t, S, X3);
  mont_mul<F>(Y3, M, t);
  fe_add<F>(t, YYYY, YYYY);
  fe_add<F>(t, t, t);
  fe_add<F>(t, t, t);
  fe_sub<F>(Y3, Y3, t);
  fe_copy<F>(R.X, X3);
  fe_copy<F>(R.Y, Y3);
  fe_copy<F>(R.Z, Z3);
}

// Shared tail of the additions: given U1, S1, H = U2 - U1, r = S2 - S1 and
// Z3 / H, X3 = r^2 - H^3 - 2 U1 H^2, Y3 = r (U1 H^2 - X3) - S1 H^3.
// Out of line: one copy per curve for the kernels that call it from many places.
template <class C>
__device__ __noinline__ void jac_dbl(Jac<typename C::Fp>& R, const Jac<typename C::Fp>& P) {
  jac_dbl_inl<C>(R, P);
}

template <class C>
ECC_DEV void jac_add_tail(Jac<typename C::Fp>& R, const uint32_t* U1, const uint32_t* S1,
                          const uint32_t* H, const uint32_t* r, const uint32_t* Z3) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  uint32_t HH[N], HHH[N], V[N], X3[N], Y3[N], t[N];
  mont_sqr<F>(HH, H);
  mont_mul<F>(HHH, H, HH);
  mont_mul<F>(V, U1, HH);
  mont_sqr<F>(X3, r);
  fe_sub<F>(X3, X3, HHH);
  fe_sub<F>(X3, X3, V);
  fe_sub<F>(X3, X3, V);
  fe_sub<F>(t, V, X3);
  mont_mul<F>(Y3, r, t);
  mont_mul<F>(t, S1, HHH);
  fe_sub<F>(Y3, Y3, t);
  fe_copy<F>(R.X, X3);
  fe_copy<F>(R.Y, Y3);
  fe_copy<F>(R.Z, Z3);
}

// R = P + Q, both Jacobian (every case of the group law).
template <class C>
ECC_DEV void jac_add_inl(Jac<typename C::Fp>& R, const Jac<typename C::Fp>& P,
                     const Jac<typename C::Fp>& Q) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  if (jac_is_inf<C>(P)) {
    R = Q;
    return;
  }
  if (jac_is_inf<C>(Q)) {
    R = P;
    return;
  }
  uint32_t Z1Z1[N], Z2Z2[N], U1[N], U2[N], S1[N], S2[N], H[N], r[N], Z3[N];
  mont_sqr<F>(Z1Z1, P.Z);
  mont_sqr<F>(Z2Z2, Q.Z);
  mont_mul<F>(U1, P.X, Z2Z2);
  mont_mul<F>(U2, Q.X, Z1Z1);
  mont_mul<F>(S1, Q.Z, Z2Z2);
  mont_mul<F>(S1, P.Y, S1);
  mont_mul<F>(S2, P.Z, Z1Z1);
  mont_mul<F>(S2, Q.Y, S2);
  fe_sub<F>(H, U2, U1);
  fe_sub<F>(r, S2, S1);
  if (fe_is_zero<F>(H)) {
    if (fe_is_zero<F>(r)) {
      jac_dbl<C>(R, P);
    } else {
      jac_set_inf<C>(R);
    }
    return;
  }
  mont_mul<F>(Z3, P.Z, Q.Z);
  mont_mul<F>(Z3, Z3, H);
  jac_add_tail<C>(R, U1, S1, H, r, Z3);
}

template <class C>
__device__ __noinline__ void jac_add(Jac<typename C::Fp>& R, const Jac<typename C::Fp>& P,
                                     const Jac<typename C::Fp>& Q) {
  jac_add_inl<C>(R, P, Q);
}

// R = P + (x, y) with the second operand affine ((0, 0) = O).
template <class C>
__device__ __noinline__ void jac_add_mixed(Jac<typename C::Fp>& R, const Jac<typename C::Fp>& P,
                           const uint32_t* x, const uint32_t* y) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  if (pt_is_inf<F>(x, y)) {
    R = P;
    return;
  }
  if (jac_is_inf<C>(P)) {
    jac_from_affine<C>(R, x, y);
    return;
  }
  uint32_t Z1Z1[N], U2[N], S2[N], H[N], r[N], Z3[N], U1[N], S1[N];
  mont_sqr<F>(Z1Z1, P.Z);
  mont_mul<F>(U2, x, Z1Z1);
  mont_mul<F>(S2, P.Z, Z1Z1);
  mont_mul<F>(S2, y, S2);
  fe_sub<F>(H, U2, P.X);
  fe_sub<F>(r, S2, P.Y);
  if (fe_is_zero<F>(H)) {
    if (fe_is_zero<F>(r)) {
      jac_dbl<C>(R, P);
    } else {
      jac_set_inf<C>(R);
    }
    return;
  }
  mont_mul<F>(Z3, P.Z, H);
  fe_copy<F>(U1, P.X);
  fe_copy<F>(S1, P.Y);
  jac_add_tail<C>(R, U1, S1, H, r, Z3);
}

// Jacobian -> affine (x, y) in Montgomery form, (0, 0) for O (one inversion).
template <class C>
__device__ __noinline__ void jac_to_affine(uint32_t* x, uint32_t* y, const Jac<typename C::Fp>& P) {
  using F = typename C::Fp;
  constexpr int N = F::N;
  if (jac_is_inf<C>(P)) {
    fe_set_zero<F>(x);
    fe_set_zero<F>(y);
    return;
  }
  uint32_t zi[N], zi2[N];
  fe_inv_mont<F>(zi, P.Z);
  mont_sqr<F>(zi2, zi);
  mont_mul<F>(x, P.X, zi2);
  mont_mul<F>(zi2, zi2, zi);
  mont_mul<F>(y, P.Y, zi2);
}

}  // namespace ecc
