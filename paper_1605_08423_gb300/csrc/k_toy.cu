// k_toy.cu -- the rotating-spring toy model of the SI ("A simple toy model") on
// which the SI compares its integrators: many independent trajectories, one
// thread each, FP64 throughout, state in registers for the whole run.
//
//   U(R) = k/2 (|R| - a)^2 in the plane, f = -grad U = -k (r - a) R / r.
//   Both acceleration matrices of the SI have the radial form
//     S = s_r P_r + s_t P_t,   P_r = R R^T / r^2,  P_t = I - P_r,
//   G_lambda (as printed): s_r = 1/lambda, s_t = 1;
//   H + mu G_lambda:       s_r = k + mu/lambda, s_t = k (1 - a/r) + mu  (H = k P_r + k (1 - a/r) P_t).
//   Then S^{-1} = P_r/s_r + P_t/s_t and the cumbersome term of Eq. standard is
//     Gamma_j = sum_i d_i (S^{-1})_{ji} = R_j [ (1/s_r)'/r + (1/s_r - 1/s_t)/r^2 ],
//   with (1/s_r)' = 0 for both choices (two dimensions: sum_i d_i (R_j R_i / r^2) = R_j / r^2).
//
// Schemes (z = L^{-T} xi, S(R) = L L^T, xi two Box-Muller normals from Philox
// counter (trajectory, step, 0, kToy)):
//   plain     R' = R + D f + sqrt(2 T D) xi                             (S = I)
//   standard  R' = R + D S^{-1} f + T D Gamma + sqrt(2 T D) z          (Eq. standard, gamma = 0)
//   first     y = R + sqrt(2 T D) z,
//             R' = y + D S^{-1} f - 1/2 S^{-1} [S(y) - S(R)] (y - R)   (Eq. smartMarkov)
//   fast      R' = R + D S^{-1} f + sqrt(2 T D) z
//                  - 1/2 S^{-1} [S(R_prev) - S(R)] (R_prev - R)        (Eq. finaldyn)
//   adopted   R' = R + Dt S^{-1} [f - (S(R_prev) - S(R))(R_prev - R)/(2 Db)]
//                  + sqrt(2 T Db) z                                      (Eq. finaldyn_new)
//   norogna   R' = R + D S^{-1} f + sqrt(2 T D) z                      (Eq. norogna)
// R_prev = R on the first step.  Per trajectory the kernel writes
// [x, y, sum U, sum U^2, sum |R|, polar angle travelled, status] with the sums
// over the positions after steps n_burn..n_steps-1; status = s + 1 when S(R) was
// not positive definite at step s (the trajectory stops there), else 0.
#include "common.cuh"
#include "kernels.cuh"

#include "qmcmd.h"

#include <cmath>

namespace qmc {

namespace {

constexpr uint32_t kToy = 8;   // Philox purpose word of the toy-model noise

struct Sym2 { double s11, s12, s22; };

// S at (x, y) in the radial form above (ir = 1/r, ir2 = 1/r^2); st_out receives s_t.
__device__ __forceinline__ Sym2 toy_smat(const ToyDev& p, double x, double y, double ir, double ir2, double& st_out) {
    const double st = p.s_mode == QMC_TOY_S_HG ? p.k * (1.0 - p.a * ir) + p.mu : 1.0;
    const double d = (p.sr_const - st) * ir2;
    st_out = st;
    return Sym2{fma(d * x, x, st), d * x * y, fma(d * y, y, st)};
}

// 2x2 Cholesky factor S = L L^T kept as l21 and the reciprocal diagonal
// (i11 = 1/l11, i22 = 1/l22, each one reciprocal square root); false if S is
// not positive definite.
struct Chol2 { double l21, i11, i22; };
__device__ __forceinline__ bool chol2(const Sym2& S, Chol2& c) {
    if (!(S.s11 > 0.0)) return false;
    c.i11 = rsqrt(S.s11);
    c.l21 = S.s12 * c.i11;
    const double d = S.s22 - c.l21 * c.l21;
    if (!(d > 0.0)) return false;
    c.i22 = rsqrt(d);
    return true;
}
// S u = v by the two triangular solves.
__device__ __forceinline__ void chol2_solve(const Chol2& c, double v0, double v1, double& u0, double& u1) {
    const double w0 = v0 * c.i11, w1 = (v1 - c.l21 * w0) * c.i22;
    u1 = w1 * c.i22;
    u0 = (w0 - c.l21 * u1) * c.i11;
}

__global__ void __launch_bounds__(256) toy_kernel(ToyDev p, int n_traj, const double* __restrict__ xy0,
                                                  double* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_traj) return;
    const double x0 = xy0[2 * t], y0 = xy0[2 * t + 1];
    double x = x0, y = y0;
    double xp = x, yp = y;
    double r2 = x * x + y * y, ir = rsqrt(r2), r = r2 * ir;
    double sp_st = 0.0;
    Sym2 Sp = toy_smat(p, x, y, ir, ir * ir, sp_st);      // S(R_prev), carried from step to step
    double su = 0.0, su2 = 0.0, sr = 0.0, status = 0.0;
    // Polar angle travelled: the sum of the per-step increments (each below pi in
    // magnitude) equals phi_end - phi_0 + 2 pi (net turns across the negative x
    // axis), so only the crossings are counted per step -- sign tests on the
    // y coordinates and on the cross product R x R' -- and phi comes from atan2
    // at the two ends.
    int turns = 0;
    const double D = p.delta;
    for (int s = 0; s < p.n_steps; ++s) {
        const uint4 w = philox((uint32_t)t, (uint32_t)s, 0u, kToy, p.key);
        const double u1 = u53(w.x, w.y), u2 = u53(w.z, w.w);
        const double rho = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        const double xi0 = rho * cs, xi1 = rho * sn;
        const double ir2 = ir * ir;
        const double fr = -p.k * (r - p.a) * ir;
        const double fx = fr * x, fy = fr * y;
        double xn, yn;
        Sym2 S{1.0, 0.0, 1.0};
        if (p.scheme == QMC_TOY_PLAIN) {
            xn = x + D * fx + p.amp * xi0;
            yn = y + D * fy + p.amp * xi1;
        } else {
            double st;
            S = toy_smat(p, x, y, ir, ir2, st);
            Chol2 c;
            if (!chol2(S, c)) { status = s + 1; break; }
            const double z1 = xi1 * c.i22, z0 = (xi0 - c.l21 * z1) * c.i11;
            double sfx, sfy;
            chol2_solve(c, fx, fy, sfx, sfy);
            switch (p.scheme) {
            case QMC_TOY_STANDARD: {
                const double g = (1.0 / p.sr_const - 1.0 / st) * ir2;   // Gamma = g R
                xn = x + D * sfx + p.T * D * g * x + p.amp * z0;
                yn = y + D * sfy + p.T * D * g * y + p.amp * z1;
                break;
            }
            case QMC_TOY_FIRST: {
                const double ex = p.amp * z0, ey = p.amp * z1;          // y - R
                const double qx = x + ex, qy = y + ey;
                const double iq = rsqrt(qx * qx + qy * qy);
                double sty;
                const Sym2 Sy = toy_smat(p, qx, qy, iq, iq * iq, sty);
                const double vx = (Sy.s11 - S.s11) * ex + (Sy.s12 - S.s12) * ey;
                const double vy = (Sy.s12 - S.s12) * ex + (Sy.s22 - S.s22) * ey;
                double wx, wy;
                chol2_solve(c, vx, vy, wx, wy);
                xn = qx + D * sfx - 0.5 * wx;
                yn = qy + D * sfy - 0.5 * wy;
                break;
            }
            case QMC_TOY_FAST:
            case QMC_TOY_ADOPTED: {
                const double ex = xp - x, ey = yp - y;                  // R_prev - R
                const double vx = (Sp.s11 - S.s11) * ex + (Sp.s12 - S.s12) * ey;
                const double vy = (Sp.s12 - S.s12) * ex + (Sp.s22 - S.s22) * ey;
                double wx, wy;
                chol2_solve(c, vx, vy, wx, wy);
                if (p.scheme == QMC_TOY_FAST) {
                    xn = x + D * sfx + p.amp * z0 - 0.5 * wx;
                    yn = y + D * sfy + p.amp * z1 - 0.5 * wy;
                } else {
                    xn = x + p.dt * (sfx - p.half_idb * wx) + p.ampb * z0;
                    yn = y + p.dt * (sfy - p.half_idb * wy) + p.ampb * z1;
                }
                break;
            }
            default:   // QMC_TOY_NOROGNA
                xn = x + D * sfx + p.amp * z0;
                yn = y + D * sfy + p.amp * z1;
                break;
            }
        }
        {
            const bool up = __double_as_longlong(y) >= 0, upn = __double_as_longlong(yn) >= 0;
            if (up != upn) {
                const long long cr = __double_as_longlong(x * yn - y * xn);
                if (up && cr > 0) ++turns;            // counter-clockwise across the negative x axis
                else if (!up && cr < 0) --turns;      // clockwise across it
            }
        }
        xp = x; yp = y; Sp = S;
        x = xn; y = yn;
        r2 = x * x + y * y;
        ir = rsqrt(r2);
        r = r2 * ir;
        if (s >= p.n_burn) {
            const double d = r - p.a;
            const double u = 0.5 * p.k * d * d;
            su += u; su2 += u * u; sr += r;
        }
    }
    const double theta = atan2(y, x) - atan2(y0, x0) + 2.0 * kPi * turns;
    double* o = out + 7 * (size_t)t;
    o[0] = x; o[1] = y; o[2] = su; o[3] = su2; o[4] = sr; o[5] = theta; o[6] = status;
}

}  // namespace

void launch_toy(const ToyDev& p, int n_traj, const double* xy0, double* out, cudaStream_t st) {
    if (n_traj <= 0) return;
    toy_kernel<<<(n_traj + 255) / 256, 256, 0, st>>>(p, n_traj, xy0, out);
}

}  // namespace qmc

// ---------------------------------------------------------------------------
// C ABI (include/qmcmd.h)
// ---------------------------------------------------------------------------
namespace {

int toy_check(const qmc_toy_params* p, int n_traj) {
    if (!p || n_traj < 0) return QMC_ERR_INVALID;
    if (p->scheme < QMC_TOY_PLAIN || p->scheme > QMC_TOY_NOROGNA) return QMC_ERR_INVALID;
    if (p->s_mode != QMC_TOY_S_G && p->s_mode != QMC_TOY_S_HG) return QMC_ERR_INVALID;
    if (!(p->delta > 0) || !(p->lambda > 0) || p->T < 0 || p->alpha < 0 || !(p->k >= 0)) return QMC_ERR_INVALID;
    if (p->n_steps < 0 || p->n_burn < 0 || p->n_burn > p->n_steps) return QMC_ERR_INVALID;
    return QMC_OK;
}

qmc::ToyDev toy_dev(const qmc_toy_params* p) {
    qmc::ToyDev d;
    d.k = p->k; d.a = p->a; d.mu = p->mu;
    d.sr_const = p->s_mode == QMC_TOY_S_HG ? p->k + p->mu / p->lambda : 1.0 / p->lambda;
    d.T = p->T; d.delta = p->delta;
    d.dt = p->delta; d.db = p->delta;
    if (p->scheme == QMC_TOY_ADOPTED && p->alpha > 0) {
        d.dt = (1.0 - std::exp(-p->alpha * p->delta)) / p->alpha;
        d.db = (1.0 - std::exp(-2.0 * p->alpha * p->delta)) / (2.0 * p->alpha);
    }
    d.half_idb = 1.0 / (2.0 * d.db);
    d.amp = std::sqrt(2.0 * p->T * p->delta);
    d.ampb = std::sqrt(2.0 * p->T * d.db);
    d.scheme = p->scheme; d.s_mode = p->s_mode; d.n_steps = p->n_steps; d.n_burn = p->n_burn;
    d.key = qmc::make_key(p->seed);
    return d;
}

}  // namespace

extern "C" int qmc_toy_langevin_device(const qmc_toy_params* p, int n_traj, const double* xy0_dev, double* out_dev,
                                       void* stream) {
    const int rc = toy_check(p, n_traj);
    if (rc != QMC_OK) return rc;
    if (n_traj > 0 && (!xy0_dev || !out_dev)) return QMC_ERR_INVALID;
    qmc::launch_toy(toy_dev(p), n_traj, xy0_dev, out_dev, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

extern "C" int qmc_toy_langevin(const qmc_toy_params* p, int n_traj, const double* xy0, double* out) {
    const int rc = toy_check(p, n_traj);
    if (rc != QMC_OK) return rc;
    if (n_traj == 0) return QMC_OK;
    if (!xy0 || !out) return QMC_ERR_INVALID;
    double *d_xy = nullptr, *d_out = nullptr;
    const size_t bxy = sizeof(double) * 2 * (size_t)n_traj, bout = sizeof(double) * QMC_TOY_NOUT * (size_t)n_traj;
    if (cudaMalloc(&d_xy, bxy) != cudaSuccess) return QMC_ERR_OOM;
    if (cudaMalloc(&d_out, bout) != cudaSuccess) { cudaFree(d_xy); return QMC_ERR_OOM; }
    int res = QMC_OK;
    if (cudaMemcpy(d_xy, xy0, bxy, cudaMemcpyHostToDevice) != cudaSuccess) res = QMC_ERR_CUDA;
    if (res == QMC_OK) {
        qmc::launch_toy(toy_dev(p), n_traj, d_xy, d_out, nullptr);
        if (cudaGetLastError() != cudaSuccess || cudaMemcpy(out, d_out, bout, cudaMemcpyDeviceToHost) != cudaSuccess)
            res = QMC_ERR_CUDA;
    }
    cudaFree(d_xy);
    cudaFree(d_out);
    if (res != QMC_OK) return res;
    for (int t = 0; t < n_traj; ++t)
        if (out[QMC_TOY_NOUT * (size_t)t + 6] != 0.0) return QMC_ERR_NOT_PD;
    return QMC_OK;
}
