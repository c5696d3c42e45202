/*
 * ORACLE for the H^2 matrix-vector product y = A^H x.
 *
 * Test infrastructure only: tests, the package's smoke check and the bench's
 * CPU baseline call it; the CUDA library never does. It shares no code, header
 * or helper with the CUDA path.
 *
 * Plain FP64, straightforward loops, one step per equation of the paper:
 *   leaf projection   xhat^q_j = V_j^T x(j)                       (Sec. 4.2, Alg. 2)
 *   upsweep           xhat^{l-1}_p = sum_c F_c^T xhat^l_c          (Eq. 2, Alg. 2)
 *   coupling          yhat^l_i = sum_{j in b_i} S^l_ij xhat^l_j    (Eq. 3, Alg. 3)
 *   downsweep         yhat^l_c += E_c yhat^{l-1}_p                 (Eq. 5, Alg. 4)
 *   leaf expansion    y(i) = U_i yhat^q_i                          (Eq. 4, Alg. 4)
 *   dense blocks      y(i) += sum_j D_ij x(j)                      (Sec. 2.2, Sec. 4.1)
 * OpenMP only splits independent nodes/rows of one step across threads.
 *
 * Input format (every block column-major):
 *   complete binary cluster tree of depth q in heap order (root 0, children
 *   2h+1, 2h+2; level l = nodes 2^l-1 .. 2^(l+1)-2; leaves = level q);
 *   leaf_offset[2^q+1]; U, V: leaf i is size_i x k at +leaf_offset[i]*k;
 *   E, F: node h>=1 is k x k at +(h-1)*k*k; S: block rows over all nodes,
 *   S_colidx = heap index of the column node, block b at +b*k*k;
 *   D: block rows over leaves, D_colidx = leaf index, block b (size_i x size_j)
 *   at +D_valoff[b].
 *
 * `mutate` != 0 plants one deliberate mistake (a transposed operand, a dropped
 * term, a wrong sign or index) so that tests can show the pins catch it.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum {
  MUT_NONE = 0,
  MUT_F_TRANSPOSED = 1,     /* upsweep applies F_c instead of F_c^T */
  MUT_E_TRANSPOSED = 2,     /* downsweep applies E_c^T instead of E_c */
  MUT_NO_DOWNSWEEP = 3,     /* parent contributions never pushed down */
  MUT_S_TRANSPOSED = 4,     /* coupling applies S_ij^T */
  MUT_NO_DENSE = 5,         /* dense near-field dropped */
  MUT_ONE_CHILD = 6,        /* upsweep sums only the first child */
  MUT_D_TRANSPOSED = 7,     /* dense block read row-major */
  MUT_DOWNSWEEP_SIGN = 8,   /* downsweep subtracts */
  MUT_COUPLING_ROW_X = 9,   /* coupling multiplies xhat of the row node */
  MUT_V_ROWMAJOR = 10,      /* leaf projection reads V row-major */
  MUT_SKIP_TOP_LEVEL = 11,  /* coupling skips the shallowest non-empty level */
};

static int node_level(int64_t h) {
  int l = 0;
  while (((int64_t)2 << l) - 1 <= h) l++;
  return l;
}

/*
 * y = A^H x for nv columns (x: n x nv, leading dim ldx; y: n x nv, leading dim ldy).
 * leaf_mask: NULL, or one byte per leaf; when given only the marked leaves' rows of
 * y are computed (the rest of y is left untouched) and the coupling/downsweep run
 * only on their ancestors. Returns 0, or -1 on allocation failure.
 */
int oracle_matvec(int64_t n, int q, int k, const int64_t* leaf_offset, const double* U, const double* V,
                  const double* E, const double* F, const int32_t* S_rowptr, const int32_t* S_colidx,
                  const double* S_val, const int32_t* D_rowptr, const int32_t* D_colidx, const int64_t* D_valoff,
                  const double* D_val, int nv, const double* x, int64_t ldx, double* y, int64_t ldy,
                  const uint8_t* leaf_mask, int mutate) {
  (void)n;
  const int64_t leaves = (int64_t)1 << q, n_nodes = ((int64_t)2 << q) - 1, leaf0 = leaves - 1;
  const int64_t kk = (int64_t)k * k;
  double* xhat = (double*)calloc((size_t)(n_nodes * nv * k), sizeof(double));
  double* yhat = (double*)calloc((size_t)(n_nodes * nv * k), sizeof(double));
  uint8_t* need = (uint8_t*)calloc((size_t)n_nodes, 1);
  if (!xhat || !yhat || !need) { free(xhat); free(yhat); free(need); return -1; }
#define XH(h, v) (xhat + ((int64_t)(h) * nv + (v)) * k)
#define YH(h, v) (yhat + ((int64_t)(h) * nv + (v)) * k)

  /* rows whose yhat is needed: ancestors (and selves) of the selected leaves */
  for (int64_t i = 0; i < leaves; i++)
    if (!leaf_mask || leaf_mask[i])
      for (int64_t h = leaf0 + i;; h = (h - 1) / 2) { need[h] = 1; if (h == 0) break; }

  /* leaf projection: xhat_j = V_j^T x(j) */
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < leaves; j++) {
    const int64_t off = leaf_offset[j], s = leaf_offset[j + 1] - off;
    const double* Vj = V + off * k;
    for (int v = 0; v < nv; v++) {
      double* xh = XH(leaf0 + j, v);
      for (int nu = 0; nu < k; nu++) {
        double acc = 0.0;
        for (int64_t a = 0; a < s; a++) {
          double vv = (mutate == MUT_V_ROWMAJOR) ? Vj[(int64_t)nu + k * a] : Vj[a + s * nu];
          acc += vv * x[off + a + ldx * v];
        }
        xh[nu] = acc;
      }
    }
  }

  /* upsweep, level by level (Eq. 2): xhat_p = F_c1^T xhat_c1 + F_c2^T xhat_c2 */
  for (int l = q; l >= 1; l--) {
    const int64_t pfirst = ((int64_t)1 << (l - 1)) - 1, pcount = (int64_t)1 << (l - 1);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < pcount; t++) {
      const int64_t p = pfirst + t;
      for (int v = 0; v < nv; v++) {
        double* xp = XH(p, v);
        for (int nu = 0; nu < k; nu++) xp[nu] = 0.0;
        for (int ci = 1; ci <= 2; ci++) {
          if (mutate == MUT_ONE_CHILD && ci == 2) continue;
          const int64_t c = 2 * p + ci;
          const double* Fc = F + (c - 1) * kk;
          const double* xc = XH(c, v);
          for (int nu = 0; nu < k; nu++) {
            double acc = 0.0;
            for (int mu = 0; mu < k; mu++) {
              double f = (mutate == MUT_F_TRANSPOSED) ? Fc[nu + (int64_t)k * mu] : Fc[mu + (int64_t)k * nu];
              acc += f * xc[mu];
            }
            xp[nu] += acc;
          }
        }
      }
    }
  }

  /* coupling, every level (Eq. 3): yhat_i = sum_j S_ij xhat_j */
  int top_level = -1;
  if (mutate == MUT_SKIP_TOP_LEVEL)
    for (int64_t h = 0; h < n_nodes && top_level < 0; h++)
      if (S_rowptr[h + 1] > S_rowptr[h]) top_level = node_level(h);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n_nodes; i++) {
    if (!need[i]) continue;
    if (mutate == MUT_SKIP_TOP_LEVEL && node_level(i) == top_level) continue;
    for (int v = 0; v < nv; v++) {
      double* yi = YH(i, v);
      for (int32_t b = S_rowptr[i]; b < S_rowptr[i + 1]; b++) {
        const int64_t j = (mutate == MUT_COUPLING_ROW_X) ? i : S_colidx[b];
        const double* Sb = S_val + (int64_t)b * kk;
        const double* xj = XH(j, v);
        for (int nu = 0; nu < k; nu++) {
          double acc = 0.0;
          for (int mu = 0; mu < k; mu++) {
            double s = (mutate == MUT_S_TRANSPOSED) ? Sb[mu + (int64_t)k * nu] : Sb[nu + (int64_t)k * mu];
            acc += s * xj[mu];
          }
          yi[nu] += acc;
        }
      }
    }
  }

  /* downsweep, level by level (Eq. 5): yhat_c += E_c yhat_p */
  if (mutate != MUT_NO_DOWNSWEEP) {
    for (int l = 1; l <= q; l++) {
      const int64_t cfirst = ((int64_t)1 << l) - 1, ccount = (int64_t)1 << l;
#pragma omp parallel for schedule(static)
      for (int64_t t = 0; t < ccount; t++) {
        const int64_t c = cfirst + t, p = (c - 1) / 2;
        if (!need[c]) continue;
        const double* Ec = E + (c - 1) * kk;
        for (int v = 0; v < nv; v++) {
          double* yc = YH(c, v);
          const double* yp = YH(p, v);
          for (int mu = 0; mu < k; mu++) {
            double acc = 0.0;
            for (int nu = 0; nu < k; nu++) {
              double e = (mutate == MUT_E_TRANSPOSED) ? Ec[nu + (int64_t)k * mu] : Ec[mu + (int64_t)k * nu];
              acc += e * yp[nu];
            }
            yc[mu] += (mutate == MUT_DOWNSWEEP_SIGN) ? -acc : acc;
          }
        }
      }
    }
  }

  /* leaf expansion (Eq. 4) then dense near-field blocks */
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < leaves; i++) {
    if (leaf_mask && !leaf_mask[i]) continue;
    const int64_t off = leaf_offset[i], s = leaf_offset[i + 1] - off;
    const double* Ui = U + off * k;
    for (int v = 0; v < nv; v++) {
      double* yv = y + ldy * v + off;
      const double* yh = YH(leaf0 + i, v);
      for (int64_t a = 0; a < s; a++) {
        double acc = 0.0;
        for (int nu = 0; nu < k; nu++) acc += Ui[a + s * nu] * yh[nu];
        yv[a] = acc;
      }
      if (mutate == MUT_NO_DENSE) continue;
      for (int32_t b = D_rowptr[i]; b < D_rowptr[i + 1]; b++) {
        const int64_t j = D_colidx[b];
        const int64_t offj = leaf_offset[j], sj = leaf_offset[j + 1] - offj;
        const double* Db = D_val + D_valoff[b];
        const double* xj = x + ldx * v + offj;
        for (int64_t a = 0; a < s; a++) {
          double acc = 0.0;
          for (int64_t c = 0; c < sj; c++) {
            double d = (mutate == MUT_D_TRANSPOSED) ? Db[c + sj * a] : Db[a + s * c];
            acc += d * xj[c];
          }
          yv[a] += acc;
        }
      }
    }
  }
#undef XH
#undef YH
  free(xhat); free(yhat); free(need);
  return 0;
}

/* number of OpenMP threads the oracle will use */
int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}
