// Objective evaluation that performs no device allocation.
//
// Some callers cannot call cudaMalloc: code running under a framework or
// serving runtime whose allocator owns the device memory (a caching
// allocator or a fixed memory pool sized at start-up, which must account for
// every byte), and code on a latency path where cudaMalloc's implicit device
// synchronisation is not acceptable.  For them, pet_objective_noalloc keeps
// its reduction scratch in a fixed array in this library's own device memory
// instead of asking for a buffer.
//
// The scratch is the file-scope array below.  Host code cannot use its name
// as a device address, so the entry point looks the address up with
// cudaGetSymbolAddress once per device (the first call on each device does
// this, with that device current) and passes the pointer to the kernels.
#include <mutex>

#include "petvr_internal.cuh"

namespace petvr {
namespace {

// Block partials of the log-likelihood and penalty reductions: 1 MiB,
// held on every device that loads the library until the process exits.
constexpr int kNoallocPartials = 131072;
static __device__ __align__(256) double g_noalloc_partials[kNoallocPartials];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double *g_setup_ptr[kMaxDevices] = {};

// The plan's tables live on plan->device, so the call must run there: the
// current device has to be the plan's (else PET_ERR_INVALID), and the scratch
// address is that device's.
pet_status scratch_for_plan_device(const pet_plan *plan, double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(PET_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev != plan->device)
        return set_error(PET_ERR_INVALID, "pet_objective_noalloc: the current device (" + std::to_string(dev) +
                                              ") is not the plan's device (" + std::to_string(plan->device) + ")");
    if (dev < 0 || dev >= kMaxDevices) return set_error(PET_ERR_INVALID, "device index beyond the supported range");
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_setup_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p)
            return set_error(PET_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_setup_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_setup_ptr[dev];
    return PET_OK;
}

}  // namespace
}  // namespace petvr

using namespace petvr;

extern "C" pet_status pet_objective_noalloc(const pet_plan *plan, const float *d_img, const float *d_counts,
                                            const float *d_bg, float bg, float beta, double *d_phi,
                                            void *stream) {
    if (!plan || !d_img || !d_counts || !d_phi) return set_error(PET_ERR_INVALID, "null argument");
    if (!(beta >= 0.0f) || !std::isfinite(beta)) return set_error(PET_ERR_INVALID, "beta must be >= 0");
    if (!std::isfinite(bg)) return set_error(PET_ERR_INVALID, "background must be finite");
    if (plan->ring) return set_error(PET_ERR_INVALID, "pet_objective_noalloc: multi-ring plans are not supported");
    // the band-chunk count of pet_objective's full-data pass, so that every
    // ray's expected count is the one pet_objective computes
    const int group = full_group(plan);
    const int n_ll = forward_blocks(plan->M, plan->nz, group);
    const long long plane = (long long)plan->N * plan->nz;
    const long long n_pen = (plane + 255) / 256;
    if ((long long)n_ll + n_pen > kNoallocPartials)
        return set_error(PET_ERR_INVALID, "pet_objective_noalloc: image/sinogram too large for its fixed scratch (" +
                                              std::to_string((long long)n_ll + n_pen) + " block partials needed, " +
                                              std::to_string(kNoallocPartials) + " available)");
    double *scratch = nullptr;
    const pet_status st = scratch_for_plan_device(plan, &scratch);
    if (st != PET_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // every block writes its own partial, so nothing has to be cleared first
    FwdArgs a{};
    a.views = plan->d_views;
    a.uc = plan->d_uc;
    a.order = plan->d_natural;
    a.v_begin = 0;
    a.v_end = plan->na;
    a.nx = plan->nx;
    a.ny = plan->ny;
    a.nz = plan->nz;
    a.nb = plan->nb;
    a.img = d_img;
    a.g = d_counts;
    a.w = d_bg;
    a.w_scalar = bg;
    a.ll_partials = scratch;
    const pet_status fs = launch_forward(a, FWD_NONE, true, group, s, nullptr);
    if (fs != PET_OK) return fs;
    return launch_objective_finish_raw(plan->nx, plan->ny, plan->nz, beta, d_img, n_ll, scratch, d_phi, s);
}
