/* Oracle helper (test infrastructure only): y = H x in the tensor-product form
 * Y = A X + X B^T + U * docc o X of the Hubbard Hamiltonian (Eq. 1), for
 * x viewed as a D_up x D_dn row-major matrix (combined index of Sec. III).
 *
 * A and B are the single-spin hopping matrices in CSR form, built by the Python
 * oracle from the sorted per-spin lists by binary search.  This file only
 * evaluates the products with plain loops (OpenMP over rows); the terms of each
 * output are added in the order: diagonal, spin-up hops (CSR order), spin-down
 * hops (CSR order).
 */
#include <stdint.h>

void oracle_kron_apply(int64_t Du, int64_t Dd,
                       const int64_t *Aptr, const int64_t *Acol, const double *Aval,
                       const int64_t *Bptr, const int64_t *Bcol, const double *Bval,
                       const uint64_t *up_str, const uint64_t *dn_str, double U,
                       const double *x, double *y)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t u = 0; u < Du; ++u) {
        const double *xu = x + u * Dd;
        double *yu = y + u * Dd;
        for (int64_t d = 0; d < Dd; ++d)
            yu[d] = U * (double)__builtin_popcountll(up_str[u] & dn_str[d]) * xu[d];
        for (int64_t k = Aptr[u]; k < Aptr[u + 1]; ++k) {
            const double a = Aval[k];
            const double *xr = x + Acol[k] * Dd;
            for (int64_t d = 0; d < Dd; ++d)
                yu[d] += a * xr[d];
        }
        for (int64_t d = 0; d < Dd; ++d) {
            double acc = yu[d];
            for (int64_t k = Bptr[d]; k < Bptr[d + 1]; ++k)
                acc += Bval[k] * xu[Bcol[k]];
            yu[d] = acc;
        }
    }
}
