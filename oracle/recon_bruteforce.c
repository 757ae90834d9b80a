/*
 * Oracle A -- the reconstruction formula written out (test infrastructure).
 *
 * ORACLE: test infrastructure only.  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline leg may load or call this file.  It shares no code
 * with the CUDA library.
 *
 * Definition (Eq. reconstruction, Sec. II-A, with the factor 1/2 per cut that
 * the single-wire identity  rho = 1/2 sum_{s in I,X,Y,Z} Tr(s rho) s  carries):
 *
 *     P(x) = 2^{-|E|}  sum_{e in {I,X,Y,Z}^{|E|}}  prod_{j=1..m}  T_j[e|E_j][x|out_j]
 *
 * For every requested state x the code loops over all 4^{|E|} cut
 * assignments e in mixed-radix order (cut 0 the fastest digit), multiplies
 * the m tensor entries selected by (e, x), and accumulates with Kahan
 * summation in FP64.  No reordering of the sum, no reuse between terms.
 *
 * Tensor layout (shared input format): node j holds n_out[j] output bits and
 * n_cut[j] cut axes; element [c_0][c_1]...[c_{n_cut-1}][x] sits at
 * ((c_0*4 + c_1)*4 + ...)*2^{n_out} + x, and bit k of x is the value of
 * original qubit out_qubits_j[k].  Basis index 0..3 = I, X, Y, Z.
 *
 * States are n-bit strings given as (lo, hi) 64-bit words (qubit q is bit q).
 *
 * `mutation` plants a known mistake (used only by the tests that show the
 * pins catch mistakes): 0 none; 1 drop the 2^{-|E|} factor; 2 skip the
 * Z basis term; 4 read output bits in reversed order; 8 read the cut axes of
 * each node in reversed order; 16 negate the X terms.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAX_CUTS 40

static int state_bit(uint64_t lo, uint64_t hi, int q) {
    return q < 64 ? (int)((lo >> q) & 1u) : (int)((hi >> (q - 64)) & 1u);
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int oracle_recon(int n_qubits, int n_nodes, int n_cuts,
                 const int *n_out, const int *out_qubits,   /* concatenated per node */
                 const int *n_cut, const int *cut_ids,      /* concatenated per node */
                 const double *const *data,
                 int64_t n_states, const uint64_t *states_lo, const uint64_t *states_hi,
                 double *out, int n_threads, int mutation) {
    if (n_cuts < 0 || n_cuts > ORACLE_MAX_CUTS || n_nodes <= 0 || n_nodes > 64 || n_qubits <= 0 ||
        n_qubits > 128)
        return -1;
    int *out_off = (int *)calloc((size_t)n_nodes + 1, sizeof(int));
    int *cut_off = (int *)calloc((size_t)n_nodes + 1, sizeof(int));
    if (!out_off || !cut_off) { free(out_off); free(cut_off); return -2; }
    for (int j = 0; j < n_nodes; ++j) {
        out_off[j + 1] = out_off[j] + n_out[j];
        cut_off[j + 1] = cut_off[j] + n_cut[j];
    }
    (void)n_threads;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t s = 0; s < n_states; ++s) {
        uint64_t lo = states_lo[s], hi = states_hi ? states_hi[s] : 0;
        int64_t xj[64];
        int e[ORACLE_MAX_CUTS];
        for (int j = 0; j < n_nodes; ++j) {
            int64_t x = 0;
            int no = n_out[j];
            for (int k = 0; k < no; ++k) {
                int kk = (mutation & 4) ? (no - 1 - k) : k;
                x |= (int64_t)state_bit(lo, hi, out_qubits[out_off[j] + kk]) << k;
            }
            xj[j] = x;
        }
        memset(e, 0, sizeof(e));
        double sum = 0.0, comp = 0.0;
        int64_t n_terms = (int64_t)1 << (2 * n_cuts);
        for (int64_t t = 0; t < n_terms; ++t) {
            int skip = 0;
            if (mutation & 2) {
                for (int c = 0; c < n_cuts; ++c) if (e[c] == 3) { skip = 1; break; }
            }
            if (!skip) {
                double term = 1.0;
                for (int j = 0; j < n_nodes; ++j) {
                    int64_t idx = 0;
                    int nc = n_cut[j];
                    for (int d = 0; d < nc; ++d) {
                        int dd = (mutation & 8) ? (nc - 1 - d) : d;
                        idx = idx * 4 + e[cut_ids[cut_off[j] + dd]];
                    }
                    term *= data[j][(idx << n_out[j]) + xj[j]];
                }
                if (mutation & 16) {
                    for (int c = 0; c < n_cuts; ++c) if (e[c] == 1) term = -term;
                }
                /* Kahan summation */
                double y = term - comp;
                double tt = sum + y;
                comp = (tt - sum) - y;
                sum = tt;
            }
            /* next assignment: cut 0 is the fastest digit */
            for (int c = 0; c < n_cuts; ++c) {
                if (++e[c] < 4) break;
                e[c] = 0;
            }
        }
        out[s] = (mutation & 1) ? sum : ldexp(sum, -n_cuts);
    }
    free(out_off);
    free(cut_off);
    return 0;
}
