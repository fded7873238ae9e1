/*
 * Oracle O1 helper — test infrastructure only, never part of the product path.
 *
 * Cyclic-by-row Jacobi eigenvalue iteration for a dense real symmetric matrix,
 * written from the textbook method (Golub & Van Loan, "Matrix Computations",
 * symmetric Schur decomposition by plane rotations). Plain FP64, no blocking.
 *
 * It diagonalises the generalised Laplacian L = L~ + rho v v^T of Def. 2.2 /
 * Def. 2.3 so that the oracle has the eigenvector basis X of Theorem 3.1 by
 * definition rather than through the Cauchy factorisation.
 */
#include <math.h>
#include <string.h>

/* a: n*n row-major symmetric input (overwritten, ends near-diagonal)
 * vec: n*n row-major output; column k is the eigenvector of w[k]
 * w: n eigenvalues (unsorted, in the order of the diagonal)
 * Returns the number of sweeps used, or -1 if max_sweeps was reached. */
int oracle_jacobi_eigh(int n, double *a, double *vec, double *w,
                       int max_sweeps, double rel_tol)
{
    memset(vec, 0, sizeof(double) * (size_t)n * (size_t)n);
    for (int i = 0; i < n; ++i) vec[(size_t)i * n + i] = 1.0;

    double fro = 0.0;
    for (size_t i = 0; i < (size_t)n * n; ++i) fro += a[i] * a[i];
    fro = sqrt(fro);
    if (fro == 0.0) {
        for (int i = 0; i < n; ++i) w[i] = 0.0;
        return 0;
    }

    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += 2.0 * a[(size_t)p * n + q] * a[(size_t)p * n + q];
        if (sqrt(off) <= rel_tol * fro) break;

        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = a[(size_t)p * n + q];
                if (apq == 0.0) continue;
                double app = a[(size_t)p * n + p];
                double aqq = a[(size_t)q * n + q];
                /* rotation angle: t = tan(phi) is the smaller root of t^2 + 2 theta t - 1 = 0 */
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0);
                double s = t * c;
                /* A <- J^T A J with J = [[c, s], [-s, c]] in the (p, q) plane */
                for (int k = 0; k < n; ++k) {
                    double akp = a[(size_t)k * n + p];
                    double akq = a[(size_t)k * n + q];
                    a[(size_t)k * n + p] = c * akp - s * akq;
                    a[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = a[(size_t)p * n + k];
                    double aqk = a[(size_t)q * n + k];
                    a[(size_t)p * n + k] = c * apk - s * aqk;
                    a[(size_t)q * n + k] = s * apk + c * aqk;
                }
                a[(size_t)p * n + q] = 0.0;
                a[(size_t)q * n + p] = 0.0;
                /* V <- V J */
                for (int k = 0; k < n; ++k) {
                    double vkp = vec[(size_t)k * n + p];
                    double vkq = vec[(size_t)k * n + q];
                    vec[(size_t)k * n + p] = c * vkp - s * vkq;
                    vec[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    for (int i = 0; i < n; ++i) w[i] = a[(size_t)i * n + i];
    return sweep < max_sweeps ? sweep : -1;
}
