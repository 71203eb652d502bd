/*
 * FP64 CPU oracle for the Pauli-rotation statevector path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library; the product path never
 * does.  It shares no code, header or table with the CUDA library.
 *
 * A plain statevector simulator in complex<double> (C99 `double complex`).
 * Conventions (paper, Sec. "Multi-qubit rotations in a fullstate simulator"):
 * amplitude index k, qubit j = bit j of k (qubit 0 least significant).
 * Pauli strings come as symplectic masks: X on x&~z, Z on z&~x, Y on x&z.
 *
 * Every multi-qubit rotation exp(-i theta/2 P) is applied the textbook way the
 * paper describes for the gate-decomposed baseline (Sec. "Preliminaries of
 * Hamiltonian Simulation", CNOT-staircase figure): a basis change on every X or
 * Y qubit of the support, a CNOT ladder that gathers the parity of the support
 * onto its highest qubit, Rz(theta) there, the ladder undone, the basis change
 * undone.  Pauli gates are applied as gates.  Nothing here uses the pair rule
 * of the method itself, so the two are checked against each other.
 *
 * Gate matrices are those of the paper's Eqs. for the Pauli matrices and for
 * H, S and CNOT (Sec. "Pauli and Clifford Group"); Rz(theta) =
 * diag(e^{-i theta/2}, e^{+i theta/2}) = exp(-i theta Z / 2).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cx;

/* parallelise only states large enough to amortise the fork */
#define PAR_MIN_QUBITS 14

static inline uint64_t insert_zero(uint64_t t, int q)
{
    uint64_t low = t & ((1ULL << q) - 1ULL);
    return ((t >> q) << (q + 1)) | low;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Thread count for later calls (timing only: single-thread and all-core rates
 * of the same oracle); k <= 0 restores one thread per processor. */
void orc_set_num_threads(int k)
{
#ifdef _OPENMP
    omp_set_num_threads(k > 0 ? k : omp_get_num_procs());
#else
    (void)k;
#endif
}

/* ---- one-qubit gates ------------------------------------------------------ */

void orc_gate_x(cx *a, int n, int q)
{
    int64_t half = (int64_t)1 << (n - 1);
    uint64_t b = 1ULL << q;
#pragma omp parallel for schedule(static) if (n >= PAR_MIN_QUBITS)
    for (int64_t t = 0; t < half; ++t) {
        uint64_t k0 = insert_zero((uint64_t)t, q), k1 = k0 | b;
        cx v = a[k0];
        a[k0] = a[k1];
        a[k1] = v;
    }
}

/* Y|0> = i|1>, Y|1> = -i|0> */
void orc_gate_y(cx *a, int n, int q)
{
    int64_t half = (int64_t)1 << (n - 1);
    uint64_t b = 1ULL << q;
#pragma omp parallel for schedule(static) if (n >= PAR_MIN_QUBITS)
    for (int64_t t = 0; t < half; ++t) {
        uint64_t k0 = insert_zero((uint64_t)t, q), k1 = k0 | b;
        cx v0 = a[k0], v1 = a[k1];
        a[k0] = -I * v1;
        a[k1] = I * v0;
    }
}

void orc_gate_z(cx *a, int n, int q)
{
    int64_t half = (int64_t)1 << (n - 1);
    uint64_t b = 1ULL << q;
#pragma omp parallel for schedule(static) if (n >= PAR_MIN_QUBITS)
    for (int64_t t = 0; t < half; ++t) {
        uint64_t k1 = insert_zero((uint64_t)t, q) | b;
        a[k1] = -a[k1];
    }
}

void orc_gate_h(cx *a, int n, int q)
{
    const double r = 1.0 / sqrt(2.0);
    int64_t half = (int64_t)1 << (n - 1);
    uint64_t b = 1ULL << q;
#pragma omp parallel for schedule(static) if (n >= PAR_MIN_QUBITS)
    for (int64_t t = 0; t < half; ++t) {
        uint64_t k0 = insert_zero((uint64_t)t, q), k1 = k0 | b;
        cx v0 = a[k0], v1 = a[k1];
        a[k0] = r * (v0 + v1);
        a[k1] = r * (v0 - v1);
    }
}

/* S = diag(1, i); Sdg = diag(1, -i) */
static void phase_one(cx *a, int n, int q, cx ph)
{
    int64_t half = (int64_t)1 << (n - 1);
    uint64_t b = 1ULL << q;
#pragma omp parallel for schedule(static) if (n >= PAR_MIN_QUBITS)
    for (int64_t t = 0; t < half; ++t) {
        uint64_t k1 = insert_zero((uint64_t)t, q) | b;
        a[k1] *= ph;
    }
}

void orc_gate_s(cx *a, int n, int q) { phase_one(a, n, q, I); }
void orc_gate_sdg(cx *a, int n, int q) { phase_one(a, n, q, -I); }

/* Rz(theta) = diag(e^{-i theta/2}, e^{+i theta/2}) */
void orc_gate_rz(cx *a, int n, int q, double theta)
{
    cx p0 = cexp(-I * 0.5 * theta), p1 = cexp(I * 0.5 * theta);
    int64_t half = (int64_t)1 << (n - 1);
    uint64_t b = 1ULL << q;
#pragma omp parallel for schedule(static) if (n >= PAR_MIN_QUBITS)
    for (int64_t t = 0; t < half; ++t) {
        uint64_t k0 = insert_zero((uint64_t)t, q), k1 = k0 | b;
        a[k0] *= p0;
        a[k1] *= p1;
    }
}

/* ---- two-qubit gate ------------------------------------------------------- */

/* CNOT(c, t): flip qubit t where qubit c is 1 */
void orc_gate_cnot(cx *a, int n, int c, int t)
{
    int64_t quarter = (int64_t)1 << (n - 2);
    int lo = c < t ? c : t, hi = c < t ? t : c;
    uint64_t bc = 1ULL << c, bt = 1ULL << t;
#pragma omp parallel for schedule(static) if (n >= PAR_MIN_QUBITS)
    for (int64_t s = 0; s < quarter; ++s) {
        uint64_t k = insert_zero(insert_zero((uint64_t)s, lo), hi) | bc;
        cx v = a[k];
        a[k] = a[k | bt];
        a[k | bt] = v;
    }
}

/* ---- Pauli strings -------------------------------------------------------- */

/* P applied as one-qubit Pauli gates (the string has no extra phase: Y is the
 * Pauli matrix Y on every Y position). */
void orc_apply_pauli(cx *a, int n, uint64_t x, uint64_t z)
{
    for (int q = 0; q < n; ++q) {
        int xb = (int)((x >> q) & 1ULL), zb = (int)((z >> q) & 1ULL);
        if (xb && zb)
            orc_gate_y(a, n, q);
        else if (xb)
            orc_gate_x(a, n, q);
        else if (zb)
            orc_gate_z(a, n, q);
    }
}

/* Gate counts of the decomposition below (for the 2(k-1) CNOT check). */
void orc_rotation_gate_count(uint64_t x, uint64_t z, int n, int *n_cnot, int *n_basis, int *n_rz)
{
    int k = 0, b = 0;
    for (int q = 0; q < n; ++q) {
        if (((x | z) >> q) & 1ULL)
            ++k;
        if ((x >> q) & 1ULL)
            b += ((z >> q) & 1ULL) ? 4 : 2; /* Y: Sdg,H ... H,S ; X: H ... H */
    }
    *n_cnot = k > 0 ? 2 * (k - 1) : 0;
    *n_basis = b;
    *n_rz = k > 0 ? 1 : 0;
}

/*
 * exp(-i theta/2 P) by the CNOT staircase.  With B = H for X and B = H.Sdg for
 * Y (so that B^dag Z B is X or Y respectively), P = B^dag (Z..Z) B, and
 * exp(-i theta/2 Z..Z) = L^dag Rz_top(theta) L with L the CNOT ladder over the
 * support in ascending qubit order.  The identity string is a global phase.
 */
void orc_rotation(cx *a, int n, uint64_t x, uint64_t z, double theta)
{
    int sup[64];
    int k = 0;
    for (int q = 0; q < n; ++q)
        if (((x | z) >> q) & 1ULL)
            sup[k++] = q;
    if (k == 0) {
        cx ph = cexp(-I * 0.5 * theta);
        int64_t dim = (int64_t)1 << n;
#pragma omp parallel for schedule(static) if (n >= PAR_MIN_QUBITS)
        for (int64_t i = 0; i < dim; ++i)
            a[i] *= ph;
        return;
    }
    for (int m = 0; m < k; ++m) {
        int q = sup[m];
        int xb = (int)((x >> q) & 1ULL), zb = (int)((z >> q) & 1ULL);
        if (xb && zb) {
            orc_gate_sdg(a, n, q);
            orc_gate_h(a, n, q);
        } else if (xb) {
            orc_gate_h(a, n, q);
        }
    }
    for (int m = 0; m + 1 < k; ++m)
        orc_gate_cnot(a, n, sup[m], sup[m + 1]);
    orc_gate_rz(a, n, sup[k - 1], theta);
    for (int m = k - 2; m >= 0; --m)
        orc_gate_cnot(a, n, sup[m], sup[m + 1]);
    for (int m = 0; m < k; ++m) {
        int q = sup[m];
        int xb = (int)((x >> q) & 1ULL), zb = (int)((z >> q) & 1ULL);
        if (xb && zb) {
            orc_gate_h(a, n, q);
            orc_gate_s(a, n, q);
        } else if (xb) {
            orc_gate_h(a, n, q);
        }
    }
}

void orc_apply_rotations(cx *a, int n, const uint64_t *x, const uint64_t *z,
                         const double *theta, int64_t count)
{
    for (int64_t j = 0; j < count; ++j)
        orc_rotation(a, n, x[j], z[j], theta[j]);
}

/*
 * A mixed sequence: kind[j] == 0 is the rotation (x[j], z[j], theta[j]);
 * kind[j] == 1 is the Pauli gate given by the masks (x[j], z[j]).
 */
void orc_apply_sequence(cx *a, int n, const int *kind, const uint64_t *x, const uint64_t *z,
                        const double *theta, int64_t count)
{
    for (int64_t j = 0; j < count; ++j) {
        if (kind[j] == 0)
            orc_rotation(a, n, x[j], z[j], theta[j]);
        else
            orc_apply_pauli(a, n, x[j], z[j]);
    }
}

/* ---- reductions ------------------------------------------------------------ */

double orc_norm2(const cx *a, int n)
{
    int64_t dim = (int64_t)1 << n;
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static) if (n >= PAR_MIN_QUBITS)
    for (int64_t i = 0; i < dim; ++i)
        s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return s;
}

/* <a|b> = sum conj(a_k) b_k */
void orc_inner(const cx *a, const cx *b, int n, double *re, double *im)
{
    int64_t dim = (int64_t)1 << n;
    double sr = 0.0, si = 0.0;
#pragma omp parallel for reduction(+ : sr, si) schedule(static) if (n >= PAR_MIN_QUBITS)
    for (int64_t i = 0; i < dim; ++i) {
        cx v = conj(a[i]) * b[i];
        sr += creal(v);
        si += cimag(v);
    }
    *re = sr;
    *im = si;
}

/*
 * <a| sum_j c_j P_j |a> (paper, Sec. "Extraction of Expectation Values"):
 * each P_j is applied gate-wise to a copy held in `work` (2^n amplitudes,
 * caller-owned), then the inner product is taken.  Returns the real part; the
 * imaginary part (zero for Hermitian P_j) is summed into *imag_out if non-NULL.
 */
double orc_expval(const cx *a, int n, const uint64_t *x, const uint64_t *z, const double *c,
                  int64_t count, cx *work, double *imag_out)
{
    size_t bytes = sizeof(cx) * ((size_t)1 << n);
    double e = 0.0, ei = 0.0;
    for (int64_t j = 0; j < count; ++j) {
        memcpy(work, a, bytes);
        orc_apply_pauli(work, n, x[j], z[j]);
        double re, im;
        orc_inner(a, work, n, &re, &im);
        e += c[j] * re;
        ei += c[j] * im;
    }
    if (imag_out)
        *imag_out = ei;
    return e;
}

/* sum_j c_j P_j |a>  into out (work as above) */
void orc_apply_pauli_sum(const cx *a, int n, const uint64_t *x, const uint64_t *z, const double *c,
                         int64_t count, cx *out, cx *work)
{
    int64_t dim = (int64_t)1 << n;
    size_t bytes = sizeof(cx) * ((size_t)dim);
    memset(out, 0, bytes);
    for (int64_t j = 0; j < count; ++j) {
        memcpy(work, a, bytes);
        orc_apply_pauli(work, n, x[j], z[j]);
        double cj = c[j];
#pragma omp parallel for schedule(static) if (n >= PAR_MIN_QUBITS)
        for (int64_t i = 0; i < dim; ++i)
            out[i] += cj * work[i];
    }
}
