// Host-side constant tables: Wigner-3j symbols, the translation coupling
// constants a5/b5 of App. I-C (Eqs. tran_coeff) and the planar class tables used
// by the apply kernels.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace tmat {

static long double lfact(int n) {
  long double r = 1.0L;
  for (int i = 2; i <= n; ++i) r *= (long double)i;
  return r;
}

// Wigner 3j symbol (j1 j2 j3; m1 m2 m3) by Racah's single-sum formula in long
// double (orders here stay <= 12, so every factorial is exact in the mantissa).
double wigner3j_host(int j1, int j2, int j3, int m1, int m2, int m3) {
  if (m1 + m2 + m3 != 0) return 0.0;
  if (j3 < std::abs(j1 - j2) || j3 > j1 + j2) return 0.0;
  if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m3) > j3) return 0.0;
  if (m1 == 0 && m2 == 0 && ((j1 + j2 + j3) & 1)) return 0.0;  // exact selection rule
  long double tri = lfact(j1 + j2 - j3) * lfact(j1 - j2 + j3) * lfact(-j1 + j2 + j3) / lfact(j1 + j2 + j3 + 1);
  long double pre = std::sqrt(tri * lfact(j1 + m1) * lfact(j1 - m1) * lfact(j2 + m2) * lfact(j2 - m2) *
                              lfact(j3 + m3) * lfact(j3 - m3));
  int kmin = std::max(0, std::max(j2 - j3 - m1, j1 - j3 + m2));
  int kmax = std::min(j1 + j2 - j3, std::min(j1 - m1, j2 + m2));
  long double sum = 0.0L;
  for (int k = kmin; k <= kmax; ++k) {
    long double den = lfact(k) * lfact(j3 - j2 + k + m1) * lfact(j3 - j1 + k - m2) * lfact(j1 + j2 - j3 - k) *
                      lfact(j1 - k - m1) * lfact(j2 - k + m2);
    sum += ((k & 1) ? -1.0L : 1.0L) / den;
  }
  int e = j1 - j2 - m3;
  long double sign = (((e % 2) + 2) % 2) ? -1.0L : 1.0L;
  return (double)(sign * pre * sum);
}

// i^e for integer e as (re, im)
static void ipow(int e, double* re, double* im) {
  int r = ((e % 4) + 4) % 4;
  const double tr[4] = {1, 0, -1, 0}, ti[4] = {0, 1, 0, -1};
  *re = tr[r];
  *im = ti[r];
}

// a5(l,m|l',m'|q), b5(l,m|l',m'|q): the coupling constants of Eqs. tran_coeff
// (summation order q; denominator 2 l(l+1) l'(l'+1); beta's second 3j symbol at
// q-1). Returned as complex numbers (the i-power included).
void coupling_a5b5(int l, int m, int lp, int mp, int q, double2* a, double2* b) {
  double ir, ii;
  ipow(std::abs(m - mp) - std::abs(m) - std::abs(mp) + lp - l + q, &ir, &ii);
  double sgn = (((m - mp) % 2) != 0) ? -1.0 : 1.0;
  double f1 = std::sqrt((2.0 * l + 1) * (2.0 * lp + 1) / (2.0 * l * (l + 1) * lp * (lp + 1)));
  double w1 = wigner3j_host(l, lp, q, m, -mp, mp - m);
  double fa = (l * (l + 1.0) + lp * (lp + 1.0) - q * (q + 1.0)) * std::sqrt(2.0 * q + 1);
  double va = sgn * f1 * fa * w1 * wigner3j_host(l, lp, q, 0, 0, 0);
  double arg = (double)(l + lp + 1 + q) * (l + lp + 1 - q) * (q + l - lp) * (q - l + lp) * (2 * q + 1);
  double vb = 0.0;
  if (q >= 1 && arg > 0) vb = sgn * f1 * std::sqrt(arg) * w1 * wigner3j_host(l, lp, q - 1, 0, 0, 0);
  a->x = va * ir;
  a->y = va * ii;
  b->x = vb * ir;
  b->y = vb * ii;
}

// Normalised associated Legendre function at x = 0:
// Pbar_q^mu(0) = sqrt((2q+1)/2 (q-mu)!/(q+mu)!) P_q^mu(0), no Condon-Shortley phase,
// by the three-term recurrence in q at x = 0.
double pbar_at_zero(int q, int mu) {
  if (mu > q) return 0.0;
  long double pmm = 1.0L;
  for (int i = 1; i < 2 * mu; i += 2) pmm *= i;
  pmm *= std::sqrt((2.0L * mu + 1) / 2.0L / lfact(2 * mu));
  long double p2 = 0.0L, p1 = pmm;
  for (int l = mu + 1; l <= q; ++l) {
    long double a = std::sqrt((4.0L * l * l - 1) / ((long double)l * l - (long double)mu * mu));
    long double b = std::sqrt(((l - 1.0L) * (l - 1.0L) - (long double)mu * mu) / (4.0L * (l - 1.0L) * (l - 1.0L) - 1));
    long double pn = -a * b * p2;  // x = 0
    p2 = p1;
    p1 = pn;
  }
  return (double)p1;
}

static int l_of(int n) {
  int l = 1;
  while ((l + 1) * (l + 1) - 1 <= n) ++l;
  return l;
}

static void build_host(Tables* t, int nmax, std::vector<double2>& a5, std::vector<double2>& b5) {
  const int L = nmax * (nmax + 2), P = 2 * L, Q = 2 * nmax + 1;
  t->nmax = nmax;
  t->L = L;
  t->P = P;
  t->Q = Q;
  std::vector<int> fl(P), fm(P), fp(P);
  for (int p = 0; p < 2; ++p)
    for (int l = 1; l <= nmax; ++l)
      for (int m = -l; m <= l; ++m) {
        int f = p * L + l * (l + 1) + m - 1;
        fl[f] = l;
        fm[f] = m;
        fp[f] = p;
      }
  t->perm.assign(P, -1);
  t->mval.assign(P, 0);
  int cnt[2] = {0, 0};
  for (int f = 0; f < P; ++f) {
    int c = ((fl[f] + fm[f] + fp[f]) % 2 + 2) % 2;
    t->perm[c * L + cnt[c]] = f;
    t->mval[c * L + cnt[c]] = fm[f];
    cnt[c]++;
  }
  // full coupling constants [n][n'][q], n = (l,m), n' = (l',m')
  a5.assign((size_t)L * L * Q, make_double2(0, 0));
  b5.assign((size_t)L * L * Q, make_double2(0, 0));
  for (int n = 0; n < L; ++n)
    for (int np = 0; np < L; ++np) {
      int l = l_of(n), m = n + 1 - l * (l + 1);
      int lp = l_of(np), mp = np + 1 - lp * (lp + 1);
      for (int q = std::abs(l - lp); q <= l + lp; ++q) {
        if (std::abs(m - mp) > q) continue;
        double2 a, b;
        coupling_a5b5(l, m, lp, mp, q, &a, &b);
        a5[((size_t)n * L + np) * Q + q] = a;
        b5[((size_t)n * L + np) * Q + q] = b;
      }
    }
  // planar class triples
  for (int op = 0; op < 2; ++op) {
    std::vector<int>& seg = t->seg[op];
    std::vector<int>& tri_idx = t->tri_idx[op];
    std::vector<double>& tri_val = t->tri_val[op];
    seg.assign((size_t)P * (Q + 1) + 1, 0);
    tri_idx.clear();
    tri_val.clear();
    for (int c = 0; c < 2; ++c)
      for (int u = 0; u < L; ++u) {
        int f = t->perm[c * L + u];
        int l = fl[f], m = fm[f], p = fp[f];
        int n = l * (l + 1) + m - 1;
        for (int q = 0; q < Q; ++q) {
          seg[(size_t)(c * L + u) * (Q + 1) + q] = (int)tri_idx.size();
          for (int up = 0; up < L; ++up) {
            int f2 = t->perm[c * L + up];
            int l2 = fl[f2], m2 = fm[f2], p2 = fp[f2];
            int n2 = l2 * (l2 + 1) + m2 - 1;
            double re, im;
            int mu;
            if (op == 0) {
              // forward: A[n, n'] = xi_{n' n}(d) = e^{i(m'-m) phi} sum_q c5(l',m'|l,m|q) h_q Pbar_q^{|m'-m|}(0)
              mu = m2 - m;
              double2 v = (p == p2) ? a5[((size_t)n2 * L + n) * Q + q] : b5[((size_t)n2 * L + n) * Q + q];
              re = v.x;
              im = v.y;
            } else {
              // adjoint: (A^T)[n, n'] = xi_{n n'}(-d) = (-1)^{m-m'} e^{i(m-m') phi} sum_q c5(l,m|l',m'|q) h_q Pbar(0)
              mu = m - m2;
              double2 v = (p == p2) ? a5[((size_t)n * L + n2) * Q + q] : b5[((size_t)n * L + n2) * Q + q];
              double s = (std::abs(mu) % 2) ? -1.0 : 1.0;
              re = s * v.x;
              im = s * v.y;
            }
            if ((q + std::abs(mu)) & 1) continue;  // Pbar_q^{|mu|}(0) = 0
            double pz = pbar_at_zero(q, std::abs(mu));
            re *= pz;
            im *= pz;
            if (re == 0.0 && im == 0.0) continue;
            // alpha entries are real, beta entries imaginary (exactly): keep one factor
            bool imag = (p != p2);
            tri_idx.push_back(up | (imag ? (1 << 15) : 0));
            tri_val.push_back(imag ? im : re);
          }
        }
      }
    // entry (c*L+u)*(Q+1) + Q closes order Q-1 of row (c,u)
    for (int cu = 0; cu < P; ++cu) {
      size_t next = (size_t)(cu + 1) * (Q + 1);
      seg[(size_t)cu * (Q + 1) + Q] = (cu + 1 < P) ? seg[next] : (int)tri_idx.size();
    }
    seg[(size_t)P * (Q + 1)] = (int)tri_idx.size();
    t->n_tri[op] = (int)tri_idx.size();
  }
  // pair-sum tables: the triples of output o = c*L+u regrouped by combination
  // a = q(q+1)/2 + (mu+q)/2 of the weights H[q, mu] = w h_q e^{i mu phi}, with
  // mu = m' - m (forward) or m - m' (adjoint) and column c*L+u' of Z
  for (int op = 0; op < 2; ++op) {
    std::vector<int>& zseg = t->zseg[op];
    std::vector<int>& zidx = t->zidx[op];
    std::vector<double>& zval = t->zval[op];
    zseg.assign((size_t)P + 1, 0);
    zidx.clear();
    zval.clear();
    for (int cu = 0; cu < P; ++cu) {
      const int c = cu / L, u = cu % L;
      zseg[cu] = (int)zidx.size();
      for (int q = 0; q < Q; ++q)
        for (int e = t->seg[op][(size_t)cu * (Q + 1) + q]; e < t->seg[op][(size_t)cu * (Q + 1) + q + 1]; ++e) {
          const int up = t->tri_idx[op][e] & 0x7fff;
          const int im = (t->tri_idx[op][e] >> 15) & 1;
          const int mu = op == 0 ? t->mval[c * L + up] - t->mval[c * L + u] : t->mval[c * L + u] - t->mval[c * L + up];
          const int a = q * (q + 1) / 2 + (mu + q) / 2;  // q + |mu| is even and |mu| <= q for every triple
          zidx.push_back((c * L + up) | (a << 8) | (im << 16));
          zval.push_back(t->tri_val[op][e]);
        }
    }
    zseg[P] = (int)zidx.size();
  }
  // pair-sum tables off the plane (no class split): every pair (n, n') of the full block
  // with its 3-D coupling constant, combination a = q^2 + mu + q of the weights
  // H[q, mu] = w h_q Pbar_q^{|mu|}(cos theta) e^{i mu phi} of d = x_i - x_j, output and
  // column in the internal order. Forward (A x)_f = sum xi_{f' f}(d) x_f': c5(n'|n|q),
  // mu = m' - m; adjoint (A^T z)_f = sum xi_{f f'}(-d) z_f': c5(n|n'|q) (-1)^q, mu = m - m'
  // (H(-d)[q, mu] = (-1)^q H(d)[q, mu]); c5 = a5 for equal polarisations, b5 otherwise,
  // each a real number times a power of i.
  for (int op = 0; op < 2; ++op) {
    std::vector<int>& zseg = t->z3seg[op];
    std::vector<int>& zidx = t->z3idx[op];
    std::vector<double>& zval = t->z3val[op];
    zseg.assign((size_t)P + 1, 0);
    zidx.clear();
    zval.clear();
    for (int o = 0; o < P; ++o) {
      zseg[o] = (int)zidx.size();
      const int f = t->perm[o], p = fp[f], l = fl[f], m = fm[f], n = l * (l + 1) + m - 1;
      for (int o2 = 0; o2 < P; ++o2) {
        const int f2 = t->perm[o2], p2 = fp[f2], l2 = fl[f2], m2 = fm[f2], n2 = l2 * (l2 + 1) + m2 - 1;
        for (int q = std::abs(l - l2); q <= l + l2; ++q) {
          const int mu = op == 0 ? m2 - m : m - m2;
          if (std::abs(mu) > q) continue;
          const size_t at = op == 0 ? ((size_t)n2 * L + n) * Q + q : ((size_t)n * L + n2) * Q + q;
          double2 v = (p == p2) ? a5[at] : b5[at];
          if (op == 1 && (q & 1)) {
            v.x = -v.x;
            v.y = -v.y;
          }
          if (v.x == 0.0 && v.y == 0.0) continue;
          const bool imag = v.x == 0.0;  // a real coupling constant times 1 or i (up to sign)
          const int a = q * q + mu + q;
          zidx.push_back(o2 | (a << 8) | ((imag ? 1 : 0) << 16));
          zval.push_back(imag ? v.y : v.x);
        }
      }
    }
    zseg[P] = (int)zidx.size();
  }
}

template <typename T>
static int upload(tmat_ctx* ctx, const std::vector<T>& v, T** out) {
  size_t bytes = std::max<size_t>(1, v.size()) * sizeof(T);
  TM_CUDA(ctx, cudaMalloc((void**)out, bytes));
  if (!v.empty()) TM_CUDA(ctx, cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return TMAT_OK;
}

int get_tables(tmat_ctx* ctx, int nmax, Tables** out) {
  if (nmax < 1 || nmax > TMAT_NMAX_MAX)
    return set_error(ctx, TMAT_EINVAL, "nmax %d outside 1..%d", nmax, TMAT_NMAX_MAX);
  auto it = ctx->tables.find(nmax);
  if (it != ctx->tables.end()) {
    *out = it->second;
    return TMAT_OK;
  }
  Tables* t = new Tables();
  std::vector<double2> a5, b5;
  build_host(t, nmax, a5, b5);
  int rc = TMAT_OK;
  do {
    if ((rc = upload(ctx, t->perm, &t->d_perm))) break;
    if ((rc = upload(ctx, t->mval, &t->d_mval))) break;
    for (int op = 0; op < 2 && !rc; ++op) {
      std::vector<float> vf(t->zval[op].begin(), t->zval[op].end());
      if ((rc = upload(ctx, t->zseg[op], &t->d_zseg[op]))) break;
      if ((rc = upload(ctx, t->zidx[op], &t->d_zidx[op]))) break;
      if ((rc = upload(ctx, vf, &t->d_zval_f32[op]))) break;
      if ((rc = upload(ctx, t->zval[op], &t->d_zval_f64[op]))) break;
      std::vector<float> vf3(t->z3val[op].begin(), t->z3val[op].end());
      if ((rc = upload(ctx, t->z3seg[op], &t->d_z3seg[op]))) break;
      if ((rc = upload(ctx, t->z3idx[op], &t->d_z3idx[op]))) break;
      if ((rc = upload(ctx, vf3, &t->d_z3val_f32[op]))) break;
      if ((rc = upload(ctx, t->z3val[op], &t->d_z3val_f64[op]))) break;
    }
    if (rc) break;
    {
      std::vector<double2> gd((size_t)t->P * t->L * t->Q, make_double2(0, 0));
      const int L = t->L, Q = t->Q;
      for (int cu = 0; cu < t->P; ++cu)
        for (int q = 0; q < Q; ++q)
          for (int e = t->seg[0][(size_t)cu * (Q + 1) + q]; e < t->seg[0][(size_t)cu * (Q + 1) + q + 1]; ++e) {
            int up = t->tri_idx[0][e] & 0x7fff;
            bool im = (t->tri_idx[0][e] >> 15) & 1;
            double v = t->tri_val[0][e];
            gd[((size_t)cu * L + up) * Q + q] = im ? make_double2(0, v) : make_double2(v, 0);
          }
      if ((rc = upload(ctx, gd, &t->d_gdense))) break;
    }
    if ((rc = upload(ctx, a5, &t->d_a5))) break;
    if ((rc = upload(ctx, b5, &t->d_b5))) break;
  } while (0);
  if (rc) {
    free_tables(t);
    return rc;
  }
  ctx->tables[nmax] = t;
  *out = t;
  return TMAT_OK;
}

void free_tables(Tables* t) {
  if (!t) return;
  cudaFree(t->d_perm);
  cudaFree(t->d_mval);
  for (int op = 0; op < 2; ++op) {
    cudaFree(t->d_zseg[op]);
    cudaFree(t->d_zidx[op]);
    cudaFree(t->d_zval_f32[op]);
    cudaFree(t->d_zval_f64[op]);
    cudaFree(t->d_z3seg[op]);
    cudaFree(t->d_z3idx[op]);
    cudaFree(t->d_z3val_f32[op]);
    cudaFree(t->d_z3val_f64[op]);
  }
  cudaFree(t->d_gdense);
  cudaFree(t->d_a5);
  cudaFree(t->d_b5);
  delete t;
}

}  // namespace tmat
