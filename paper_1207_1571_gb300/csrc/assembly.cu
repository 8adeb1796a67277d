// assembly.cu -- finite-volume matrix assembly and corrections (paper Sec. 3
// and Sec. 4.3.3: gradient, divergence, Laplacian, the flux and velocity
// corrections), one thread per cell gathering over the cell's faces.
//
// Every face quantity is computed in the face's own orientation (owner =
// lower cell index, weight w on the owner), x_f = w x_own + (1 - w) x_nei,
// so both cells of a face obtain bit-identical face values and the pressure
// matrix is exactly symmetric; each cell then applies the sign of the face
// as seen from itself.  Face fields (phi*, a_f, ...) are written by the
// owner cell only, so no face is written twice and no atomics are needed.
//
// Discretisation (the paper follows the textbook collocated finite-volume
// PISO / SIMPLE; the terms below are that method):
//  momentum, row P:  ddt V/dt (PISO); central convection with flux F out of
//    P: diag += F w_P, off(P,N) = F w_N; diffusion D = nu |S| delta:
//    diag += D, off -= D; explicit non-orthogonal diffusion nu |S| k.grad u;
//    fixed-velocity face: src += (D_b - F_b) u_b, diag += D_b; outlet face
//    (zero-gradient): diag += F_b; SIMPLE: diag' = diag/alpha_u,
//    src += (diag' - diag) u.
//  pressure:  a_f = rAU_f |S| delta, diag += a_f, off = -a_f,
//    b = -sum_out phi* + sum_out rAU_f |S| k.grad p; outlet: diag += a_b,
//    b += a_b p_b; reference cell: b += diag p_ref, diag *= 2.
//  corrections: phi = phi* - a_f (p_N - p_P) - non-orthogonal term,
//    u = HbyA - rAU grad p.
#include "fvgb_internal.h"

namespace fvgb {

constexpr int kAsmBlock = 256;

struct MeshView {
    int N, F, B, M, nonorth;
    const int32_t *__restrict__ slice_ptr;
    const int32_t *__restrict__ col;
    const int32_t *__restrict__ sface;
    const int32_t *__restrict__ bptr;
    const int32_t *__restrict__ bface;
    const int8_t *__restrict__ btype;
    const double *__restrict__ Sf;
    const double *__restrict__ magSf;
    const double *__restrict__ w;
    const double *__restrict__ delta;
    const double *__restrict__ kv;
    const double *__restrict__ V;
    const double *__restrict__ Vinv;
};

static MeshView view(const fv_mesh *m)
{
    return MeshView{m->N, m->F, m->B, m->M, m->nonorth, m->slice_ptr, m->col, m->sface,
                    m->bptr, m->bface, m->btype, m->Sf, m->magSf, m->w, m->delta, m->kv,
                    m->V, m->Vinv};
}

static int blocks_for(int n) { return (n + kAsmBlock - 1) / kAsmBlock; }

// x with its sign flipped when neg (the face value as seen from the
// neighbour cell).  Integer operations on the sign bit: a multiply by -1
// would take the FP64 pipe, which bounds these kernels.  Bit-identical to
// (neg ? -1.0 : 1.0) * x, so every sum keeps its rounding.
__device__ __forceinline__ double with_sign(double x, bool neg)
{
    return __longlong_as_double(__double_as_longlong(x) ^ ((long long)neg << 63));
}

// ------------------------------------------------------------ momentum --

struct MomArgs {
    const double *u, *p, *phi, *ub, *pb, *gradU;
    double nu, dt_inv, alpha_u;
    const double *nu_cell;   // per-cell viscosity (batched cases) or nullptr
    double *Md, *Mo, *src, *gradp;
};

__global__ void __launch_bounds__(kAsmBlock) k_momentum(MeshView m, MomArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const size_t N = m.N;
    const int s = i >> 5;
    const int e0 = m.slice_ptr[s] + (i & 31), K = (m.slice_ptr[s + 1] - m.slice_ptr[s]) >> 5;
    const double vdt = m.V[i] * a.dt_inv;
    // both cells of a face belong to the same case, so the owner's value is
    // the face's
    const double nu = a.nu_cell ? a.nu_cell[i] : a.nu;
    double diag = vdt;
    double src0 = vdt * a.u[i], src1 = vdt * a.u[N + i], src2 = vdt * a.u[2 * N + i];
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    const double pP = a.p[i];
    for (int k = 0; k < K; ++k) {
        const int e = e0 + 32 * k;
        const int f = m.sface[e];
        if (f < 0) { a.Mo[e] = 0.0; continue; }
        const int c = m.col[e];
        const bool own = i < c;
        const int lo = own ? i : c, hi = own ? c : i;
        const double w = m.w[f];
        const double wS = own ? w : 1.0 - w;       // weight of this cell on the face
        const double wO = own ? 1.0 - w : w;       // weight of the other cell
        const double Fo = with_sign(a.phi[f], !own);   // flux out of this cell
        const double D = nu * m.magSf[f] * m.delta[f];
        diag += Fo * wS;
        diag += D;
        a.Mo[e] = Fo * wO - D;
        const double pf = with_sign(w * a.p[lo] + (1.0 - w) * a.p[hi], !own);
        g0 += m.Sf[f] * pf;
        g1 += m.Sf[m.M + f] * pf;
        g2 += m.Sf[2 * m.M + f] * pf;
        if (m.nonorth) {
            const double k0 = m.kv[f], k1 = m.kv[m.F + f], k2 = m.kv[2 * m.F + f];
            double t[3];
            for (int cc = 0; cc < 3; ++cc) {
                const double *G = a.gradU + (size_t)3 * cc * N;
                const double gx = w * G[lo] + (1.0 - w) * G[hi];
                const double gy = w * G[N + lo] + (1.0 - w) * G[N + hi];
                const double gz = w * G[2 * N + lo] + (1.0 - w) * G[2 * N + hi];
                t[cc] = nu * m.magSf[f] * (k0 * gx + k1 * gy + k2 * gz);
            }
            src0 += with_sign(t[0], !own);
            src1 += with_sign(t[1], !own);
            src2 += with_sign(t[2], !own);
        }
    }
    for (int j = m.bptr[i]; j < m.bptr[i + 1]; ++j) {
        const int b = m.bface[j];
        const int fb = m.F + b;
        const int type = m.btype[b];
        double pbv;
        if (type == FV_PATCH_OUTLET) {
            diag += a.phi[fb];
            pbv = a.pb[b];
        } else {
            const double D = nu * m.magSf[fb] * m.delta[fb];
            const double Fb = a.phi[fb];
            diag += D;
            const double u0 = a.ub[b], u1 = a.ub[m.B + b], u2 = a.ub[2 * m.B + b];
            src0 += D * u0 - Fb * u0;
            src1 += D * u1 - Fb * u1;
            src2 += D * u2 - Fb * u2;
            pbv = pP;
        }
        g0 += m.Sf[fb] * pbv;
        g1 += m.Sf[m.M + fb] * pbv;
        g2 += m.Sf[2 * m.M + fb] * pbv;
    }
    if (a.dt_inv == 0.0) {
        const double d1 = diag / a.alpha_u;
        src0 += (d1 - diag) * a.u[i];
        src1 += (d1 - diag) * a.u[N + i];
        src2 += (d1 - diag) * a.u[2 * N + i];
        diag = d1;
    }
    const double vi = m.Vinv[i];
    a.Md[i] = diag;
    a.src[i] = src0;
    a.src[N + i] = src1;
    a.src[2 * N + i] = src2;
    a.gradp[i] = g0 * vi;
    a.gradp[N + i] = g1 * vi;
    a.gradp[2 * N + i] = g2 * vi;
}

// gradient of the three velocity components (non-orthogonal meshes only)
__global__ void __launch_bounds__(kAsmBlock) k_grad_u(MeshView m, const double *__restrict__ u,
                                                      const double *__restrict__ ub,
                                                      double *__restrict__ gU)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const size_t N = m.N;
    const int s = i >> 5;
    const int e0 = m.slice_ptr[s] + (i & 31), K = (m.slice_ptr[s + 1] - m.slice_ptr[s]) >> 5;
    double g[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < K; ++k) {
        const int e = e0 + 32 * k;
        const int f = m.sface[e];
        if (f < 0) continue;
        const int c = m.col[e];
        const bool own = i < c;
        const int lo = own ? i : c, hi = own ? c : i;
        const double w = m.w[f];
        const double S0 = with_sign(m.Sf[f], !own), S1 = with_sign(m.Sf[m.M + f], !own),
                     S2 = with_sign(m.Sf[2 * m.M + f], !own);
        for (int cc = 0; cc < 3; ++cc) {
            const double uf = w * u[cc * N + lo] + (1.0 - w) * u[cc * N + hi];
            g[3 * cc] += S0 * uf;
            g[3 * cc + 1] += S1 * uf;
            g[3 * cc + 2] += S2 * uf;
        }
    }
    for (int j = m.bptr[i]; j < m.bptr[i + 1]; ++j) {
        const int b = m.bface[j];
        const int fb = m.F + b;
        const bool fixed = m.btype[b] != FV_PATCH_OUTLET;
        for (int cc = 0; cc < 3; ++cc) {
            const double ubv = fixed ? ub[cc * m.B + b] : u[cc * N + i];
            g[3 * cc] += m.Sf[fb] * ubv;
            g[3 * cc + 1] += m.Sf[m.M + fb] * ubv;
            g[3 * cc + 2] += m.Sf[2 * m.M + fb] * ubv;
        }
    }
    const double vi = m.Vinv[i];
    for (int q = 0; q < 9; ++q) gU[q * N + i] = g[q] * vi;
}

// ---------------------------------------------------------- H and rAU --

__global__ void __launch_bounds__(kAsmBlock) k_hbya(MeshView m, const double *__restrict__ Md,
                                                    const double *__restrict__ Mo,
                                                    const double *__restrict__ src,
                                                    const double *__restrict__ u,
                                                    double *__restrict__ HbyA,
                                                    double *__restrict__ rAU)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const size_t N = m.N;
    const int s = i >> 5;
    const int e0 = m.slice_ptr[s] + (i & 31), K = (m.slice_ptr[s + 1] - m.slice_ptr[s]) >> 5;
    double h0 = src[i], h1 = src[N + i], h2 = src[2 * N + i];
    for (int k = 0; k < K; ++k) {
        const int e = e0 + 32 * k;
        const double a = Mo[e];      // zero on padding entries
        const int c = m.col[e];
        h0 -= a * u[c];
        h1 -= a * u[N + c];
        h2 -= a * u[2 * N + c];
    }
    const double rec = 1.0 / Md[i];
    HbyA[i] = h0 * rec;
    HbyA[N + i] = h1 * rec;
    HbyA[2 * N + i] = h2 * rec;
    rAU[i] = m.V[i] * rec;
}

// ------------------------------------------------------------ pressure --

struct PresArgs {
    const double *HbyA, *rAU, *ub, *pb, *gradp;
    int ref;
    double p_ref;
    const int8_t *pin;       // per-cell reference flags (batched cases) or nullptr
    double *Pd, *Po, *b, *phis, *af, *nof;
};

__global__ void __launch_bounds__(kAsmBlock) k_pressure(MeshView m, PresArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const size_t N = m.N;
    const int s = i >> 5;
    const int e0 = m.slice_ptr[s] + (i & 31), K = (m.slice_ptr[s + 1] - m.slice_ptr[s]) >> 5;
    double diag = 0.0, bb = 0.0;
    for (int k = 0; k < K; ++k) {
        const int e = e0 + 32 * k;
        const int f = m.sface[e];
        if (f < 0) { a.Po[e] = 0.0; continue; }
        const int c = m.col[e];
        const bool own = i < c;
        const int lo = own ? i : c, hi = own ? c : i;
        const double w = m.w[f];
        const double S0 = m.Sf[f], S1 = m.Sf[m.M + f], S2 = m.Sf[2 * m.M + f];
        const double h0 = w * a.HbyA[lo] + (1.0 - w) * a.HbyA[hi];
        const double h1 = w * a.HbyA[N + lo] + (1.0 - w) * a.HbyA[N + hi];
        const double h2 = w * a.HbyA[2 * N + lo] + (1.0 - w) * a.HbyA[2 * N + hi];
        const double ph = h0 * S0 + h1 * S1 + h2 * S2;      // owner -> neighbour
        const double rf = w * a.rAU[lo] + (1.0 - w) * a.rAU[hi];
        const double af = rf * m.magSf[f] * m.delta[f];
        diag += af;
        a.Po[e] = -af;
        bb -= with_sign(ph, !own);
        double nf = 0.0;
        if (m.nonorth) {
            const double gx = w * a.gradp[lo] + (1.0 - w) * a.gradp[hi];
            const double gy = w * a.gradp[N + lo] + (1.0 - w) * a.gradp[N + hi];
            const double gz = w * a.gradp[2 * N + lo] + (1.0 - w) * a.gradp[2 * N + hi];
            nf = rf * m.magSf[f] * (m.kv[f] * gx + m.kv[m.F + f] * gy + m.kv[2 * m.F + f] * gz);
            bb += with_sign(nf, !own);
        }
        if (own) {
            a.phis[f] = ph;
            a.af[f] = af;
            if (m.nonorth) a.nof[f] = nf;
        }
    }
    for (int j = m.bptr[i]; j < m.bptr[i + 1]; ++j) {
        const int b = m.bface[j];
        const int fb = m.F + b;
        const double S0 = m.Sf[fb], S1 = m.Sf[m.M + fb], S2 = m.Sf[2 * m.M + fb];
        double ph;
        if (m.btype[b] == FV_PATCH_OUTLET) {
            ph = a.HbyA[i] * S0 + a.HbyA[N + i] * S1 + a.HbyA[2 * N + i] * S2;
            const double ab = a.rAU[i] * m.magSf[fb] * m.delta[fb];
            a.af[fb] = ab;
            diag += ab;
            bb += ab * a.pb[b];
        } else {
            ph = a.ub[b] * S0 + a.ub[m.B + b] * S1 + a.ub[2 * m.B + b] * S2;
        }
        a.phis[fb] = ph;
        bb -= ph;
    }
    if (i == a.ref || (a.pin && a.pin[i])) {
        bb += diag * a.p_ref;
        diag *= 2.0;
    }
    a.Pd[i] = diag;
    a.b[i] = bb;
}

// --------------------------------------------------------- corrections --

struct CorrArgs {
    const double *phis, *af, *nof, *pb, *HbyA, *rAU;
    const double *p;        // pressure used for the flux
    const double *pg;       // pressure whose gradient corrects u (may equal p)
    double *phi, *gradp, *u;
    double *prelax;         // SIMPLE: relaxed pressure out (nullptr for PISO)
    const double *pold;
    double alpha_p;
};

// PISO: flux from p, gradient of p, velocity from that gradient.
__global__ void __launch_bounds__(kAsmBlock) k_correct(MeshView m, CorrArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const size_t N = m.N;
    const int s = i >> 5;
    const int e0 = m.slice_ptr[s] + (i & 31), K = (m.slice_ptr[s + 1] - m.slice_ptr[s]) >> 5;
    const double pP = a.p[i];
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    for (int k = 0; k < K; ++k) {
        const int e = e0 + 32 * k;
        const int f = m.sface[e];
        if (f < 0) continue;
        const int c = m.col[e];
        const bool own = i < c;
        const int lo = own ? i : c, hi = own ? c : i;
        const double w = m.w[f];
        // face value as seen from this cell
        const double pf = with_sign(w * a.p[lo] + (1.0 - w) * a.p[hi], !own);
        g0 += m.Sf[f] * pf;
        g1 += m.Sf[m.M + f] * pf;
        g2 += m.Sf[2 * m.M + f] * pf;
        if (own) {
            double v = a.phis[f] - a.af[f] * (a.p[c] - pP);
            if (m.nonorth) v -= a.nof[f];
            a.phi[f] = v;
        }
    }
    for (int j = m.bptr[i]; j < m.bptr[i + 1]; ++j) {
        const int b = m.bface[j];
        const int fb = m.F + b;
        double pbv;
        if (m.btype[b] == FV_PATCH_OUTLET) {
            pbv = a.pb[b];
            a.phi[fb] = a.phis[fb] - a.af[fb] * (pbv - pP);
        } else {
            pbv = pP;
            a.phi[fb] = a.phis[fb];
        }
        g0 += m.Sf[fb] * pbv;
        g1 += m.Sf[m.M + fb] * pbv;
        g2 += m.Sf[2 * m.M + fb] * pbv;
    }
    const double vi = m.Vinv[i], r = a.rAU[i];
    g0 *= vi; g1 *= vi; g2 *= vi;
    a.gradp[i] = g0;
    a.gradp[N + i] = g1;
    a.gradp[2 * N + i] = g2;
    a.u[i] = a.HbyA[i] - r * g0;
    a.u[N + i] = a.HbyA[N + i] - r * g1;
    a.u[2 * N + i] = a.HbyA[2 * N + i] - r * g2;
}

// Gauss gradient of the pressure with its boundary values (fixed on
// outlets, zero-gradient elsewhere): the same sums as in k_correct, for the
// non-orthogonal correctors that re-evaluate the explicit term.
__global__ void __launch_bounds__(kAsmBlock) k_grad_p(MeshView m, const double *__restrict__ p,
                                                      const double *__restrict__ pb,
                                                      double *__restrict__ gradp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const size_t N = m.N;
    const int s = i >> 5;
    const int e0 = m.slice_ptr[s] + (i & 31), K = (m.slice_ptr[s + 1] - m.slice_ptr[s]) >> 5;
    const double pP = p[i];
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    for (int k = 0; k < K; ++k) {
        const int e = e0 + 32 * k;
        const int f = m.sface[e];
        if (f < 0) continue;
        const int c = m.col[e];
        const bool own = i < c;
        const int lo = own ? i : c, hi = own ? c : i;
        const double w = m.w[f];
        // face value as seen from this cell
        const double pf = with_sign(w * p[lo] + (1.0 - w) * p[hi], !own);
        g0 += m.Sf[f] * pf;
        g1 += m.Sf[m.M + f] * pf;
        g2 += m.Sf[2 * m.M + f] * pf;
    }
    for (int j = m.bptr[i]; j < m.bptr[i + 1]; ++j) {
        const int b = m.bface[j];
        const int fb = m.F + b;
        const double pbv = m.btype[b] == FV_PATCH_OUTLET ? pb[b] : pP;
        g0 += m.Sf[fb] * pbv;
        g1 += m.Sf[m.M + fb] * pbv;
        g2 += m.Sf[2 * m.M + fb] * pbv;
    }
    const double vi = m.Vinv[i];
    gradp[i] = g0 * vi;
    gradp[N + i] = g1 * vi;
    gradp[2 * N + i] = g2 * vi;
}

// SIMPLE, first half: flux from the solved pressure p, relaxed pressure
// prelax = pold + alpha_p (p - pold) (cell-local).
__global__ void __launch_bounds__(kAsmBlock) k_flux_relax(MeshView m, CorrArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const int s = i >> 5;
    const int e0 = m.slice_ptr[s] + (i & 31), K = (m.slice_ptr[s + 1] - m.slice_ptr[s]) >> 5;
    const double pP = a.p[i];
    for (int k = 0; k < K; ++k) {
        const int e = e0 + 32 * k;
        const int f = m.sface[e];
        if (f < 0) continue;
        const int c = m.col[e];
        if (i < c) {
            double v = a.phis[f] - a.af[f] * (a.p[c] - pP);
            if (m.nonorth) v -= a.nof[f];
            a.phi[f] = v;
        }
    }
    for (int j = m.bptr[i]; j < m.bptr[i + 1]; ++j) {
        const int b = m.bface[j];
        const int fb = m.F + b;
        if (m.btype[b] == FV_PATCH_OUTLET) a.phi[fb] = a.phis[fb] - a.af[fb] * (a.pb[b] - pP);
        else a.phi[fb] = a.phis[fb];
    }
    a.prelax[i] = a.pold[i] + a.alpha_p * (pP - a.pold[i]);
}

// SIMPLE, second half: gradient of the relaxed pressure, velocity.
__global__ void __launch_bounds__(kAsmBlock) k_grad_correct_u(MeshView m, CorrArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const size_t N = m.N;
    const int s = i >> 5;
    const int e0 = m.slice_ptr[s] + (i & 31), K = (m.slice_ptr[s + 1] - m.slice_ptr[s]) >> 5;
    const double *pg = a.pg;
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    for (int k = 0; k < K; ++k) {
        const int e = e0 + 32 * k;
        const int f = m.sface[e];
        if (f < 0) continue;
        const int c = m.col[e];
        const bool own = i < c;
        const int lo = own ? i : c, hi = own ? c : i;
        const double w = m.w[f];
        // face value as seen from this cell
        const double pf = with_sign(w * pg[lo] + (1.0 - w) * pg[hi], !own);
        g0 += m.Sf[f] * pf;
        g1 += m.Sf[m.M + f] * pf;
        g2 += m.Sf[2 * m.M + f] * pf;
    }
    for (int j = m.bptr[i]; j < m.bptr[i + 1]; ++j) {
        const int b = m.bface[j];
        const int fb = m.F + b;
        const double pbv = m.btype[b] == FV_PATCH_OUTLET ? a.pb[b] : pg[i];
        g0 += m.Sf[fb] * pbv;
        g1 += m.Sf[m.M + fb] * pbv;
        g2 += m.Sf[2 * m.M + fb] * pbv;
    }
    const double vi = m.Vinv[i], r = a.rAU[i];
    g0 *= vi; g1 *= vi; g2 *= vi;
    a.gradp[i] = g0;
    a.gradp[N + i] = g1;
    a.gradp[2 * N + i] = g2;
    a.u[i] = a.HbyA[i] - r * g0;
    a.u[N + i] = a.HbyA[N + i] - r * g1;
    a.u[2 * N + i] = a.HbyA[2 * N + i] - r * g2;
}

// -------------------------------------------------- SIMPLE residuals --
// Deterministic two-stage sums: per-block partials, then one block adds
// them in block order.

template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&v)[NV], double *out)
{
    __shared__ double red[NV][kAsmBlock / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < NV; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[k][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double x = 0.0;
        for (int q = 0; q < kAsmBlock / 32; ++q) x += red[threadIdx.x][q];
        out[threadIdx.x] = x;
    }
}

// momentum: ||b_c - M u_c||^2, ||b_c||^2 (c = 0..2) -> 6 values per block
__global__ void __launch_bounds__(kAsmBlock) k_resid_mom(MeshView m, const double *__restrict__ Md,
                                                         const double *__restrict__ Mo,
                                                         const double *__restrict__ src,
                                                         const double *__restrict__ gradp,
                                                         const double *__restrict__ u,
                                                         double *__restrict__ part)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v[6] = {0, 0, 0, 0, 0, 0};
    if (i < m.N) {
        const size_t N = m.N;
        const int s = i >> 5;
        const int e0 = m.slice_ptr[s] + (i & 31), K = (m.slice_ptr[s + 1] - m.slice_ptr[s]) >> 5;
        for (int cc = 0; cc < 3; ++cc) {
            const double *uc = u + cc * N;
            double ax = Md[i] * uc[i];
            for (int k = 0; k < K; ++k) {
                const int e = e0 + 32 * k;
                ax += Mo[e] * uc[m.col[e]];
            }
            const double b = src[cc * N + i] - m.V[i] * gradp[cc * N + i];
            v[2 * cc] += (b - ax) * (b - ax);
            v[2 * cc + 1] += b * b;
        }
    }
    block_reduce_store<6>(v, part + (size_t)blockIdx.x * 8);
}

// pressure: ||b - A p||^2 and ||phi*||^2 (owner side + boundary faces)
__global__ void __launch_bounds__(kAsmBlock) k_resid_p(MeshView m, const double *__restrict__ Pd,
                                                       const double *__restrict__ Po,
                                                       const double *__restrict__ pbv,
                                                       const double *__restrict__ p,
                                                       const double *__restrict__ phis,
                                                       double *__restrict__ part)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v[2] = {0, 0};
    if (i < m.N) {
        const int s = i >> 5;
        const int e0 = m.slice_ptr[s] + (i & 31), K = (m.slice_ptr[s + 1] - m.slice_ptr[s]) >> 5;
        double ax = Pd[i] * p[i];
        for (int k = 0; k < K; ++k) {
            const int e = e0 + 32 * k;
            const int c = m.col[e];
            ax += Po[e] * p[c];
            const int f = m.sface[e];
            if (f >= 0 && i < c) v[1] += phis[f] * phis[f];
        }
        for (int j = m.bptr[i]; j < m.bptr[i + 1]; ++j) {
            const double ph = phis[m.F + m.bface[j]];
            v[1] += ph * ph;
        }
        const double r = pbv[i] - ax;
        v[0] = r * r;
    }
    block_reduce_store<2>(v, part + (size_t)blockIdx.x * 8 + 6);
}

// out[0] = momentum measure, out[1] = pressure measure, out[2] = max
__global__ void k_resid_final(int nblocks, const double *__restrict__ part, double *__restrict__ out)
{
    __shared__ double acc[8][kAsmBlock];
    for (int k = 0; k < 8; ++k) {
        double x = 0.0;
        for (int j = threadIdx.x; j < nblocks; j += kAsmBlock) x += part[(size_t)j * 8 + k];
        acc[k][threadIdx.x] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[8];
        for (int k = 0; k < 8; ++k) {
            double x = 0.0;
            for (int q = 0; q < kAsmBlock; ++q) x += acc[k][q];
            t[k] = x;
        }
        double rmax = 0.0, bmax = 0.0;
        for (int cc = 0; cc < 3; ++cc) {
            rmax = fmax(rmax, sqrt(t[2 * cc]));
            bmax = fmax(bmax, sqrt(t[2 * cc + 1]));
        }
        const double rm = bmax > 0.0 ? rmax / bmax : 0.0;
        const double nr = sqrt(t[6]), nphi = sqrt(t[7]);
        const double rp = nphi > 0.0 ? nr / nphi : nr;
        out[0] = rm;
        out[1] = rp;
        out[2] = fmax(rm, rp);
    }
}

// --------------------------------------------------- utility kernels --

__global__ void k_gauss_grad(MeshView m, const double *__restrict__ x, const double *__restrict__ xb,
                             double *__restrict__ g)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const size_t N = m.N;
    const int s = i >> 5;
    const int e0 = m.slice_ptr[s] + (i & 31), K = (m.slice_ptr[s + 1] - m.slice_ptr[s]) >> 5;
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    for (int k = 0; k < K; ++k) {
        const int e = e0 + 32 * k;
        const int f = m.sface[e];
        if (f < 0) continue;
        const int c = m.col[e];
        const bool own = i < c;
        const int lo = own ? i : c, hi = own ? c : i;
        const double w = m.w[f];
        // face value as seen from this cell
        const double xf = with_sign(w * x[lo] + (1.0 - w) * x[hi], !own);
        g0 += m.Sf[f] * xf;
        g1 += m.Sf[m.M + f] * xf;
        g2 += m.Sf[2 * m.M + f] * xf;
    }
    for (int j = m.bptr[i]; j < m.bptr[i + 1]; ++j) {
        const int b = m.bface[j];
        const int fb = m.F + b;
        g0 += m.Sf[fb] * xb[b];
        g1 += m.Sf[m.M + fb] * xb[b];
        g2 += m.Sf[2 * m.M + fb] * xb[b];
    }
    const double vi = m.Vinv[i];
    g[i] = g0 * vi;
    g[N + i] = g1 * vi;
    g[2 * N + i] = g2 * vi;
}

__global__ void k_ldu_to_sell(MeshView m, const double *__restrict__ upper,
                              const double *__restrict__ lower, double *__restrict__ val)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const int s = i >> 5;
    const int e0 = m.slice_ptr[s] + (i & 31), K = (m.slice_ptr[s + 1] - m.slice_ptr[s]) >> 5;
    for (int k = 0; k < K; ++k) {
        const int e = e0 + 32 * k;
        const int f = m.sface[e];
        val[e] = f < 0 ? 0.0 : (i < m.col[e] ? upper[f] : lower[f]);
    }
}

__global__ void k_ldu_matvec(MeshView m, const double *__restrict__ diag,
                             const double *__restrict__ upper, const double *__restrict__ lower,
                             const double *__restrict__ x, double *__restrict__ y)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.N) return;
    const int s = i >> 5;
    const int e0 = m.slice_ptr[s] + (i & 31), K = (m.slice_ptr[s + 1] - m.slice_ptr[s]) >> 5;
    double acc = diag[i] * x[i];
    for (int k = 0; k < K; ++k) {
        const int e = e0 + 32 * k;
        const int f = m.sface[e];
        if (f < 0) continue;
        const int c = m.col[e];
        acc += (i < c ? upper[f] : lower[f]) * x[c];
    }
    y[i] = acc;
}

// cell fields: internal[new_of_old[i]] = original[i] (to_internal) or back
__global__ void k_permute_cells(int N, int ncomp, const int32_t *__restrict__ no,
                                const double *__restrict__ src, double *__restrict__ dst,
                                int to_internal)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int j = no[i];
    for (int c = 0; c < ncomp; ++c) {
        if (to_internal) dst[(size_t)c * N + j] = src[(size_t)c * N + i];
        else dst[(size_t)c * N + i] = src[(size_t)c * N + j];
    }
}

__global__ void k_permute_faces(int M, const int32_t *__restrict__ no, const int8_t *__restrict__ fl,
                                const double *__restrict__ src, double *__restrict__ dst,
                                int to_internal)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= M) return;
    const int g = no[f];
    const double sg = fl[f] ? -1.0 : 1.0;
    if (to_internal) dst[g] = sg * src[f];
    else dst[f] = sg * src[g];
}

// Uniform boundary value on boundary faces [start, start + n): u (if
// set_u) and p.  Values travel as kernel arguments, so the fill is
// stream-ordered, needs no host staging and can be captured in a graph.
__global__ void k_patch_fill(int B, int start, int n, int set_u, double u0, double u1, double u2,
                             double p, double *__restrict__ ub, double *__restrict__ pb)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const size_t b = (size_t)start + j;
    if (set_u) {
        ub[b] = u0;
        ub[(size_t)B + b] = u1;
        ub[2 * (size_t)B + b] = u2;
    }
    pb[b] = p;
}

// ------------------------------------------------------------ launches --

#define LAUNCH_CHECK() FV_CUDA(cudaGetLastError())

fv_status launch_grad_u(const fv_case *c)
{
    const fv_mesh *m = c->mesh;
    k_grad_u<<<blocks_for(m->N), kAsmBlock, 0, m->stream>>>(view(m), c->u, c->ub, c->gradU);
    LAUNCH_CHECK();
    return FV_OK;
}

fv_status launch_momentum(const fv_case *c, const StepArgs &s)
{
    const fv_mesh *m = c->mesh;
    MomArgs a{c->u, c->p, c->phi, c->ub, c->pb, c->gradU, c->nu, s.dt_inv, s.alpha_u,
              c->nu_cell, c->Md, c->Mo, c->src, c->gradp};
    k_momentum<<<blocks_for(m->N), kAsmBlock, 0, m->stream>>>(view(m), a);
    LAUNCH_CHECK();
    return FV_OK;
}

fv_status launch_hbya(const fv_case *c)
{
    const fv_mesh *m = c->mesh;
    k_hbya<<<blocks_for(m->N), kAsmBlock, 0, m->stream>>>(view(m), c->Md, c->Mo, c->src, c->u,
                                                          c->HbyA, c->rAU);
    LAUNCH_CHECK();
    return FV_OK;
}

fv_status launch_pressure(const fv_case *c, const StepArgs &s)
{
    const fv_mesh *m = c->mesh;
    PresArgs a{c->HbyA, c->rAU, c->ub, c->pb, c->gradp, s.ref_cell, s.p_ref, c->pin,
               c->Pd, c->Po, c->pbv, c->phis, c->af, c->nof};
    k_pressure<<<blocks_for(m->N), kAsmBlock, 0, m->stream>>>(view(m), a);
    LAUNCH_CHECK();
    return FV_OK;
}

fv_status launch_grad_p(const fv_case *c)
{
    const fv_mesh *m = c->mesh;
    k_grad_p<<<blocks_for(m->N), kAsmBlock, 0, m->stream>>>(view(m), c->p, c->pb, c->gradp);
    LAUNCH_CHECK();
    return FV_OK;
}

fv_status launch_correct_piso(const fv_case *c)
{
    const fv_mesh *m = c->mesh;
    CorrArgs a{c->phis, c->af, c->nof, c->pb, c->HbyA, c->rAU, c->p, c->p, c->phi, c->gradp,
               c->u, nullptr, nullptr, 0.0};
    k_correct<<<blocks_for(m->N), kAsmBlock, 0, m->stream>>>(view(m), a);
    LAUNCH_CHECK();
    return FV_OK;
}

fv_status launch_correct_simple(const fv_case *c, double alpha_p)
{
    const fv_mesh *m = c->mesh;
    // pold holds the pressure before the solve; the relaxed field is written
    // over it, then becomes the new p
    CorrArgs a{c->phis, c->af, c->nof, c->pb, c->HbyA, c->rAU, c->p, c->pold, c->phi, c->gradp,
               c->u, c->pold, c->pold, alpha_p};
    k_flux_relax<<<blocks_for(m->N), kAsmBlock, 0, m->stream>>>(view(m), a);
    LAUNCH_CHECK();
    k_grad_correct_u<<<blocks_for(m->N), kAsmBlock, 0, m->stream>>>(view(m), a);
    LAUNCH_CHECK();
    FV_CUDA(cudaMemcpyAsync(c->p, c->pold, sizeof(double) * m->N, cudaMemcpyDeviceToDevice,
                            m->stream));
    return FV_OK;
}

fv_status launch_simple_residuals_mom(const fv_case *c)
{
    const fv_mesh *m = c->mesh;
    k_resid_mom<<<blocks_for(m->N), kAsmBlock, 0, m->stream>>>(view(m), c->Md, c->Mo, c->src,
                                                               c->gradp, c->u, c->resid);
    LAUNCH_CHECK();
    return FV_OK;
}

fv_status launch_simple_residuals_p(const fv_case *c)
{
    const fv_mesh *m = c->mesh;
    k_resid_p<<<blocks_for(m->N), kAsmBlock, 0, m->stream>>>(view(m), c->Pd, c->Po, c->pbv, c->p,
                                                             c->phis, c->resid);
    LAUNCH_CHECK();
    k_resid_final<<<1, kAsmBlock, 0, m->stream>>>(blocks_for(m->N), c->resid, c->dsimple);
    LAUNCH_CHECK();
    return FV_OK;
}

fv_status launch_gauss_grad(const fv_mesh *m, const double *x, const double *xb, double *g)
{
    k_gauss_grad<<<blocks_for(m->N), kAsmBlock, 0, m->stream>>>(view(m), x, xb, g);
    LAUNCH_CHECK();
    return FV_OK;
}

fv_status launch_ldu_matvec(const fv_mesh *m, const double *diag, const double *upper,
                            const double *lower, const double *x, double *y)
{
    k_ldu_matvec<<<blocks_for(m->N), kAsmBlock, 0, m->stream>>>(view(m), diag, upper, lower, x, y);
    LAUNCH_CHECK();
    return FV_OK;
}

fv_status launch_ldu_to_sell(const fv_mesh *m, const double *upper, const double *lower,
                             double *val)
{
    k_ldu_to_sell<<<blocks_for(m->N), kAsmBlock, 0, m->stream>>>(view(m), upper, lower, val);
    LAUNCH_CHECK();
    return FV_OK;
}

fv_status launch_permute_cells(const fv_mesh *m, int ncomp, const double *src, double *dst,
                               int to_internal)
{
    k_permute_cells<<<blocks_for(m->N), kAsmBlock, 0, m->stream>>>(m->N, ncomp, m->cell_new_of_old,
                                                                   src, dst, to_internal);
    LAUNCH_CHECK();
    return FV_OK;
}

fv_status launch_patch_fill(const fv_case *c, int start, int n, const double *u, double p)
{
    const fv_mesh *m = c->mesh;
    if (n <= 0) return FV_OK;
    k_patch_fill<<<blocks_for(n), kAsmBlock, 0, m->stream>>>(
        m->B, start, n, u != nullptr, u ? u[0] : 0.0, u ? u[1] : 0.0, u ? u[2] : 0.0, p, c->ub, c->pb);
    LAUNCH_CHECK();
    return FV_OK;
}

fv_status launch_permute_faces(const fv_mesh *m, const double *src, double *dst, int to_internal)
{
    k_permute_faces<<<blocks_for(m->M), kAsmBlock, 0, m->stream>>>(m->M, m->face_new_of_old,
                                                                   m->flipped, src, dst, to_internal);
    LAUNCH_CHECK();
    return FV_OK;
}

}  // namespace fvgb
