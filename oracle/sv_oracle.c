/*
 * CPU ORACLE -- test infrastructure only.
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline leg
 * may load this library. The product path (the CUDA library and its binding)
 * never calls it, links it or shares code with it.
 *
 * What it computes (TensorLy-Quantum, Sec. 1 and Sec. 3, the expectation value
 * <H> of a circuit and its full gradient):
 *
 *   |psi(theta)> = U_G ... U_1 |0...0>,     E(theta) = sum_t c_t <psi|P_t|psi>,
 *
 * on a dense 2^n complex128 statevector, one gate at a time, in the order given.
 * No fusion, no blocking, no light cones. Qubit q is bit q of the index.
 *
 * Gate conventions (the paper fixes none; these are the readings used throughout):
 *   RX(a) = exp(-i a X/2) = [[c, -i s], [-i s, c]]
 *   RY(a) = exp(-i a Y/2) = [[c, -s], [s, c]]
 *   RZ(a) = exp(-i a Z/2) = diag(e^{-i a/2}, e^{+i a/2})
 *   RZZ(a) = exp(-i a Z(x)Z/2): phase e^{-i a/2} if the two bits agree, e^{+i a/2} if not
 *   CZ = diag(1, 1, 1, -1)
 * with c = cos(a/2), s = sin(a/2).
 *
 * Gradient (Sec. 3: "the full gradient calculation nabla <H>", done there by
 * backpropagation): this oracle uses its own adjoint sweep. With lambda = H psi at
 * the end and both vectors walked backwards gate by gate, a gate
 * G = exp(-i a K/2) contributes  dE/da = Im <lambda_k | K | psi_k>  where psi_k and
 * lambda_k are the two vectors just after that gate.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum { K_RX = 0, K_RY = 1, K_RZ = 2, K_RZZ = 3, K_CZ = 4 };

typedef struct {
    int32_t kind, q0, q1, param;
    double angle;
} orc_gate;

static double gate_angle(const orc_gate* g, const double* theta) {
    return g->param >= 0 ? theta[g->param] : g->angle;
}

/* Apply one gate with the given angle; sign = +1 applies G, sign = -1 applies G^dagger. */
static void apply_gate(int n, cplx* psi, const orc_gate* g, double a, int sign) {
    const int64_t N = (int64_t)1 << n;
    const double c = cos(0.5 * a), s = sin(0.5 * a) * (double)sign;
    if (g->kind == K_RX || g->kind == K_RY) {
        const int64_t m = (int64_t)1 << g->q0;
        #pragma omp parallel for schedule(static) if (N >= 65536)
        for (int64_t x = 0; x < N; ++x) {
            if (x & m) continue;
            cplx a0 = psi[x], a1 = psi[x | m];
            if (g->kind == K_RY) {
                psi[x] = c * a0 - s * a1;
                psi[x | m] = s * a0 + c * a1;
            } else {
                psi[x] = c * a0 - I * s * a1;
                psi[x | m] = -I * s * a0 + c * a1;
            }
        }
    } else if (g->kind == K_RZ) {
        const int64_t m = (int64_t)1 << g->q0;
        const cplx p0 = c - I * s, p1 = c + I * s;
        #pragma omp parallel for schedule(static) if (N >= 65536)
        for (int64_t x = 0; x < N; ++x) psi[x] *= (x & m) ? p1 : p0;
    } else if (g->kind == K_RZZ) {
        const int64_t m0 = (int64_t)1 << g->q0, m1 = (int64_t)1 << g->q1;
        const cplx same = c - I * s, diff = c + I * s;
        #pragma omp parallel for schedule(static) if (N >= 65536)
        for (int64_t x = 0; x < N; ++x) {
            int b0 = (x & m0) != 0, b1 = (x & m1) != 0;
            psi[x] *= (b0 == b1) ? same : diff;
        }
    } else { /* CZ, self-inverse */
        const int64_t m = ((int64_t)1 << g->q0) | ((int64_t)1 << g->q1);
        #pragma omp parallel for schedule(static) if (N >= 65536)
        for (int64_t x = 0; x < N; ++x)
            if ((x & m) == m) psi[x] = -psi[x];
    }
}

/* out = P psi for the Pauli string (letters over sites). */
static void apply_pauli(int n, const cplx* psi, cplx* out, int nsites, const int32_t* sites,
                        const char* letters) {
    const int64_t N = (int64_t)1 << n;
    int64_t flip = 0;
    for (int k = 0; k < nsites; ++k)
        if (letters[k] == 'X' || letters[k] == 'Y') flip |= (int64_t)1 << sites[k];
    #pragma omp parallel for schedule(static) if (N >= 65536)
    for (int64_t x = 0; x < N; ++x) {
        cplx f = 1.0;
        for (int k = 0; k < nsites; ++k) {
            int bit = (int)((x >> sites[k]) & 1);
            if (letters[k] == 'Y') f *= bit ? I : -I;
            else if (letters[k] == 'Z') f *= bit ? -1.0 : 1.0;
        }
        out[x] = f * psi[x ^ flip];
    }
}

static cplx inner(int n, const cplx* a, const cplx* b) {
    const int64_t N = (int64_t)1 << n;
    double re = 0.0, im = 0.0;
    #pragma omp parallel for reduction(+ : re, im) schedule(static) if (N >= 65536)
    for (int64_t x = 0; x < N; ++x) {
        cplx v = conj(a[x]) * b[x];
        re += creal(v);
        im += cimag(v);
    }
    return re + I * im;
}

/* |psi> = U |0...0>; psi must hold 2^n entries (written here). */
void orc_run(int n, const orc_gate* gates, int ngates, const double* theta, double* psi_ri) {
    cplx* psi = (cplx*)psi_ri;
    const int64_t N = (int64_t)1 << n;
    memset(psi, 0, sizeof(cplx) * (size_t)N);
    psi[0] = 1.0;
    for (int k = 0; k < ngates; ++k) apply_gate(n, psi, &gates[k], gate_angle(&gates[k], theta), +1);
}

/* <psi|P|psi> for one Pauli string (real up to rounding; the real part is returned). */
double orc_pauli_expectation(int n, const double* psi_ri, int nsites, const int32_t* sites,
                             const char* letters) {
    const int64_t N = (int64_t)1 << n;
    const cplx* psi = (const cplx*)psi_ri;
    cplx* tmp = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    if (!tmp) return NAN;
    apply_pauli(n, psi, tmp, nsites, sites, letters);
    double e = creal(inner(n, psi, tmp));
    free(tmp);
    return e;
}

/* Terms are given flattened: term t covers sites[off[t] .. off[t+1]) and the same
 * range of letters. Per-term expectation values are written to e_terms (nullable). */
double orc_energy(int n, const orc_gate* gates, int ngates, const double* theta, int nterms,
                  const double* coeff, const int32_t* off, const int32_t* sites, const char* letters,
                  double* e_terms) {
    const int64_t N = (int64_t)1 << n;
    double* psi = (double*)malloc(sizeof(cplx) * (size_t)N);
    if (!psi) return NAN;
    orc_run(n, gates, ngates, theta, psi);
    double E = 0.0;
    for (int t = 0; t < nterms; ++t) {
        double e = orc_pauli_expectation(n, psi, off[t + 1] - off[t], sites + off[t], letters + off[t]);
        if (e_terms) e_terms[t] = e;
        E += coeff[t] * e;
    }
    free(psi);
    return E;
}

/* Energy and the full gradient dE/dtheta_p (summed over every gate carrying p) by the
 * adjoint sweep described in the header. grad has n_params entries (overwritten).
 * Returns 0 on success, -1 on allocation failure. */
int orc_grad_adjoint(int n, const orc_gate* gates, int ngates, const double* theta, int n_params,
                     int nterms, const double* coeff, const int32_t* off, const int32_t* sites,
                     const char* letters, double* energy, double* grad) {
    const int64_t N = (int64_t)1 << n;
    cplx* psi = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    cplx* lam = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    cplx* tmp = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    if (!psi || !lam || !tmp) { free(psi); free(lam); free(tmp); return -1; }
    orc_run(n, gates, ngates, theta, (double*)psi);
    /* lambda = H psi */
    memset(lam, 0, sizeof(cplx) * (size_t)N);
    for (int t = 0; t < nterms; ++t) {
        apply_pauli(n, psi, tmp, off[t + 1] - off[t], sites + off[t], letters + off[t]);
        const double ct = coeff[t];
        #pragma omp parallel for schedule(static) if (N >= 65536)
        for (int64_t x = 0; x < N; ++x) lam[x] += ct * tmp[x];
    }
    *energy = creal(inner(n, psi, lam));
    for (int p = 0; p < n_params; ++p) grad[p] = 0.0;
    for (int k = ngates - 1; k >= 0; --k) {
        const orc_gate* g = &gates[k];
        const double a = gate_angle(g, theta);
        if (g->param >= 0) {
            /* tmp = K psi with K the gate's generator */
            int32_t s2[2] = {g->q0, g->q1};
            const char* lx = g->kind == K_RX ? "X" : g->kind == K_RY ? "Y" : g->kind == K_RZ ? "Z" : "ZZ";
            apply_pauli(n, psi, tmp, g->kind == K_RZZ ? 2 : 1, s2, lx);
            grad[g->param] += cimag(inner(n, lam, tmp));
        }
        apply_gate(n, psi, g, a, -1);
        apply_gate(n, lam, g, a, -1);
    }
    free(psi); free(lam); free(tmp);
    return 0;
}

int orc_version(void) { return 1; }
