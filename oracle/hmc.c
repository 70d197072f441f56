/*
 * hmc.c -- oracle Hamiltonian and leapfrog integrator (Sec. 2.1, Algorithm 1).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 * Pins: reversibility (negate p, integrate back), O(eps^2) energy error, and
 * the closed-form linear map of leapfrog on a quadratic target
 * (tests/test_oracle_hmc.py).
 */
#include "oracle.h"

double oracle_hamiltonian(const double* p, int64_t D, double logpi) {
    /* H = kinetic + potential = 1/2 |p|^2 - log pi(theta), identity mass. */
    double kin = 0.0;
    for (int64_t d = 0; d < D; ++d) kin += p[d] * p[d];
    return 0.5 * kin - logpi;
}

void oracle_leapfrog(const oracle_target* t, double* theta, double* p, double* grad,
                     double* logpi, double eps, int32_t steps) {
    const int64_t D = t->D;
    for (int32_t l = 0; l < steps; ++l) {
        for (int64_t d = 0; d < D; ++d) p[d] += 0.5 * eps * grad[d];   /* p_{l+1/2}  */
        for (int64_t d = 0; d < D; ++d) theta[d] += eps * p[d];         /* theta_{l+1} */
        *logpi = oracle_logpi(t, theta, grad);
        for (int64_t d = 0; d < D; ++d) p[d] += 0.5 * eps * grad[d];   /* p_{l+1}    */
    }
}
