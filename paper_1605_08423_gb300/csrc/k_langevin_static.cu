// k_langevin_static.cu -- the accelerated Langevin step of k_langevin.cu for
// callers that cannot allocate device memory.
//
// Why: cudaMalloc and cudaFree may synchronise the whole device, which a host
// that overlaps many trajectories on streams, or that runs a latency-bound MD
// loop, cannot afford; and some embedding hosts hand the library only
// pre-allocated buffers and own every other byte of device memory.  This entry
// point therefore allocates nothing: the caller passes every input and output
// as a device buffer, and the Cholesky workspace is a statically allocated
// device array of QMC_STATIC_MAX_N3^2 doubles (1.18 MB) that every GPU which
// loads the library holds until the process exits.
//
// The host cannot use the array's name as a device address, so the address is
// looked up with cudaGetSymbolAddress once per device (with that device
// current) on the first call there; make that first call before any stream
// capture.  All calls share the array: calls that overlap on the GPU (for
// example on two streams) race on it.  Each call clears the error word first;
// the workspace needs no clearing (every entry read is written earlier in the
// same call).
#include <mutex>

#include "../../include/qmcmd.h"
#include "common.cuh"
#include "langevin_core.cuh"

namespace qmc {

static __device__ __align__(256) double g_langevin_scratch[QMC_STATIC_MAX_N3 * QMC_STATIC_MAX_N3];
static __device__ __align__(256) int g_langevin_err;

// The step of langevin_kernel (same device code, cta_langevin_step), with the
// previous pair (R_prev, S_prev) given by the caller (nothing is stored) and
// the result written to Rout.  Rout may be R itself (the entry point passes
// the same buffer): R, Rprev and Rout are therefore not __restrict__, and every
// read of R and Rprev is done before the barrier that precedes the store.
__global__ void __launch_bounds__(1024) langevin_static_kernel(int n, const double* R, const double* Rprev,
                                                               const double* __restrict__ f,
                                                               const double* __restrict__ S,
                                                               const double* __restrict__ Sprev, double* Lc,
                                                               double* Rout, double T, double delta, double alpha,
                                                               Key key, uint32_t md, double box, int identity,
                                                               int* err) {
    extern __shared__ double v[];
    __shared__ double red[32];
    double* r1 = nullptr;
    if (!cta_langevin_step(n, R, Rprev, f, S, Sprev, Lc, T, delta, alpha, key, md, box, identity, kLvAdopted, v, red,
                           &r1)) {
        if (threadIdx.x == 0) atomicOr(err, kErrNotPD);
        return;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) Rout[i] = r1[i];
}

namespace {
struct StaticAddr {
    double* scratch = nullptr;
    int* err = nullptr;
};
std::mutex g_static_mutex;
StaticAddr g_static_addr[64];   // per device ordinal

// Device addresses of the static arrays on the current device (looked up once).
int static_addresses(StaticAddr* out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return QMC_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_static_mutex);
    StaticAddr& a = g_static_addr[dev];
    if (!a.scratch) {
        void* p = nullptr;
        void* e = nullptr;
        if (cudaGetSymbolAddress(&p, g_langevin_scratch) != cudaSuccess ||
            cudaGetSymbolAddress(&e, g_langevin_err) != cudaSuccess) {
            cudaGetLastError();
            return QMC_ERR_CUDA;
        }
        a.scratch = (double*)p;
        a.err = (int*)e;
    }
    *out = a;
    return QMC_OK;
}
}  // namespace

}  // namespace qmc

extern "C" int qmc_langevin_step_static(int n3, double* R, const double* Rprev, const double* f, const double* S,
                                        const double* Sprev, double T_kelvin, double delta, int s_mode, double alpha,
                                        uint64_t seed, uint32_t step, double box, void* stream) {
    using namespace qmc;
    if (n3 < 1 || n3 > QMC_STATIC_MAX_N3) return QMC_ERR_INVALID;
    if (!R || !Rprev || !f) return QMC_ERR_INVALID;
    if (s_mode != QMC_S_IDENTITY && s_mode != QMC_S_COV) return QMC_ERR_INVALID;
    if (s_mode == QMC_S_COV && (!S || !Sprev)) return QMC_ERR_INVALID;
    if (!(delta > 0) || T_kelvin < 0) return QMC_ERR_INVALID;
    StaticAddr a;
    int rc = static_addresses(&a);
    if (rc != QMC_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int identity = s_mode == QMC_S_IDENTITY;
    if (cudaMemsetAsync(a.err, 0, sizeof(int), st) != cudaSuccess) return QMC_ERR_CUDA;
    const size_t smem = 5 * (size_t)n3 * sizeof(double);
    langevin_static_kernel<<<1, 1024, smem, st>>>(n3, R, Rprev, f, S, Sprev, a.scratch, R,
                                                   T_kelvin * 3.166811563e-6, delta, identity ? 0.0 : alpha,
                                                   make_key(seed), step, box, identity, a.err);
    if (cudaGetLastError() != cudaSuccess) return QMC_ERR_CUDA;
    int e = 0;
    if (cudaMemcpyAsync(&e, a.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return QMC_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return QMC_ERR_CUDA;
    if (e & kErrNotPD) return QMC_ERR_NOT_PD;
    return QMC_OK;
}
