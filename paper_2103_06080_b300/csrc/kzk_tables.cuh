// kzk_tables.cuh -- plan-time FP64 generation of the diagonal propagators of
// Eq. 11 (E = e^z, Phi1 = (e^z - 1)/z, Phi2 = (e^z - 1 - z)/z^2) on the device.
//
// z(k_tau, k_y) = dsigma * ( -diffraction * k_y^2 / (i k_tau + reg_eps * diffraction)
//                            - A k_tau^2 + sum_r C_r (i k_tau)^2 / (1 + i theta_r k_tau) ),
// the paper's regularised multiplier (reg_eps = machine epsilon of the working
// precision) plus the optional relaxation processes.  At the tau-Nyquist
// frequency, where k_tau and -k_tau alias, the odd parts (diffraction, the
// imaginary part of relaxation) are dropped so that real fields stay real.
//
// Tables are even in k_y, so only |k_y| indices l = 0..ny/2 are stored:
// T[l][m] for m = 0..nx/2-1, with column 0 packing the two real values at
// k_tau = 0 (re) and the tau-Nyquist (im), mirroring the state layout.
// Stored scaled: E' = E/ny, P1' = dsigma Phi1/(nx ny), P2' = dsigma Phi2/(nx ny).
#pragma once
#include "kzk_common.cuh"

namespace kzk {

struct TabArgs {
    int nx, ny;
    double dt, A, diffraction, reg_eps, kts, kys;   // kts = 2 pi / tau length, kys = 2 pi / y length
    int n_relax;                                    // relaxation processes
    double relax_C[2], relax_theta[2];
    void* E;
    void* P1;
    void* P2;
    void* E_lo;      // float plans: E' - (float)E' (nullptr for double)
    void* Em1;       // compensated-state plans: (E - 1)/ny = z Phi1 / ny (nullptr otherwise)
};

// phi-functions at z.  |z| < 1/2: Phi2 from its Taylor series
// sum_k z^k / (k+2)!, Phi1 = 1 + z Phi2; otherwise Phi1 = (e^z - 1)/z with
// e^z - 1 formed without cancellation, Phi2 = (Phi1 - 1)/z.
__device__ __forceinline__ void phi_eval(double zr, double zi, double2& E, double2& P1, double2& P2)
{
    double sz, cz;
    sincos(zi, &sz, &cz);
    const double ex = exp(zr);
    E = make_double2(ex * cz, ex * sz);
    if (zr * zr + zi * zi < 0.25) {
        // Horner from k = 26 down: coefficient 1/(k+2)!
        double inv_f[27];
        double f = 1.0;
        for (int k = 0; k < 27; k++) { f /= (double)(k + 2); inv_f[k] = f; }
        double pr = inv_f[26], pi = 0.0;
        for (int k = 25; k >= 0; k--) {
            const double nr = zr * pr - zi * pi + inv_f[k];
            const double ni = zr * pi + zi * pr;
            pr = nr; pi = ni;
        }
        P2 = make_double2(pr, pi);
        P1 = make_double2(1.0 + zr * pr - zi * pi, zr * pi + zi * pr);
    } else {
        const double sh = sin(0.5 * zi);
        const double emr = expm1(zr) * cz - 2.0 * sh * sh;
        const double emi = ex * sz;
        const double d = zr * zr + zi * zi;
        // (a + ib) / z = (a + ib) conj(z) / |z|^2
        const double p1r = (emr * zr + emi * zi) / d, p1i = (emi * zr - emr * zi) / d;
        P1 = make_double2(p1r, p1i);
        const double qr = p1r - 1.0, qi = p1i;
        P2 = make_double2((qr * zr + qi * zi) / d, (qi * zr - qr * zi) / d);
    }
}

__device__ __forceinline__ double2 z_of(const TabArgs& a, double kt, double ky, bool nyquist)
{
    const double absorb = -a.A * kt * kt;
    // relaxation: C (i kt)^2 / (1 + i theta kt) = -C kt^2 (1 - i theta kt) / (1 + theta^2 kt^2)
    double rr = 0.0, ri = 0.0;
    for (int r = 0; r < a.n_relax; r++) {
        const double tk = a.relax_theta[r] * kt, g = a.relax_C[r] * kt * kt / (1.0 + tk * tk);
        rr -= g;
        ri += g * tk;
    }
    if (nyquist) return make_double2(a.dt * (absorb + rr), 0.0);
    // q = -diffraction ky^2 / (eps diffraction + i kt)
    const double dr = a.reg_eps * a.diffraction, di = kt;
    const double num = -a.diffraction * ky * ky;
    const double den = dr * dr + di * di;
    const double qr = num * dr / den, qi = -num * di / den;
    return make_double2(a.dt * (qr + absorb + rr), a.dt * (qi + ri));
}

template <typename T>
__global__ void tables_kernel(TabArgs a)
{
    const int n = a.nx / 2, nl = a.ny / 2 + 1;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nl * n) return;
    const int l = (int)(idx / n), m = (int)(idx % n);
    const double ky = a.kys * l;
    const double sE = 1.0 / a.ny, sP = a.dt / ((double)a.nx * a.ny);
    double2 E, P1, P2;
    cx<T> oE, oP1, oP2;
    if (m == 0) {
        double2 E0, P10, P20, EN, P1N, P2N;
        const double2 z0 = z_of(a, 0.0, ky, false);
        const double2 zN = z_of(a, a.kts * n, ky, true);
        phi_eval(z0.x, z0.y, E0, P10, P20);
        phi_eval(zN.x, zN.y, EN, P1N, P2N);
        oE = mk<T>((T)(E0.x * sE), (T)(EN.x * sE));
        oP1 = mk<T>((T)(P10.x * sP), (T)(P1N.x * sP));
        oP2 = mk<T>((T)(P20.x * sP), (T)(P2N.x * sP));
    } else {
        const double2 z = z_of(a, a.kts * m, ky, false);
        phi_eval(z.x, z.y, E, P1, P2);
        oE = mk<T>((T)(E.x * sE), (T)(E.y * sE));
        oP1 = mk<T>((T)(P1.x * sP), (T)(P1.y * sP));
        oP2 = mk<T>((T)(P2.x * sP), (T)(P2.y * sP));
    }
    reinterpret_cast<cx<T>*>(a.E)[idx] = oE;
    if (a.E_lo) {
        // two-float E': the lo part carries the rounding error of the hi part
        double ex, ey;
        if (m == 0) {
            double2 E0, P10, P20, EN, P1N, P2N;
            const double2 z0 = z_of(a, 0.0, ky, false);
            const double2 zN = z_of(a, a.kts * n, ky, true);
            phi_eval(z0.x, z0.y, E0, P10, P20);
            phi_eval(zN.x, zN.y, EN, P1N, P2N);
            ex = E0.x * sE; ey = EN.x * sE;
        } else {
            ex = E.x * sE; ey = E.y * sE;
        }
        reinterpret_cast<cx<T>*>(a.E_lo)[idx] = mk<T>((T)(ex - (double)oE.x), (T)(ey - (double)oE.y));
    }
    reinterpret_cast<cx<T>*>(a.P1)[idx] = oP1;
    reinterpret_cast<cx<T>*>(a.P2)[idx] = oP2;
    if (a.Em1) {
        // E - 1 = z Phi1, without the cancellation of forming E first
        cx<T> o;
        if (m == 0) {
            double2 E0, P10, P20, EN, P1N, P2N;
            const double2 z0 = z_of(a, 0.0, ky, false);
            const double2 zN = z_of(a, a.kts * n, ky, true);
            phi_eval(z0.x, z0.y, E0, P10, P20);
            phi_eval(zN.x, zN.y, EN, P1N, P2N);
            o = mk<T>((T)((z0.x * P10.x - z0.y * P10.y) * sE), (T)((zN.x * P1N.x - zN.y * P1N.y) * sE));
        } else {
            const double2 z = z_of(a, a.kts * m, ky, false);
            o = mk<T>((T)((z.x * P1.x - z.y * P1.y) * sE), (T)((z.x * P1.y + z.y * P1.x) * sE));
        }
        reinterpret_cast<cx<T>*>(a.Em1)[idx] = o;
    }
}

}  // namespace kzk
