// noalloc.cu -- a field solve that allocates no device memory.
//
// Who needs it: callers that must not allocate at the moment they solve.
// Examples are hosts that hand the library a fixed memory budget and forbid
// growth after start-up, and real-time loops where an allocation could stall
// on a device-wide synchronisation.  pic_field_solve allocates its multigrid
// workspace through a handle; pic_field_solve_noalloc runs the same FP64
// multigrid solve on the caller's device arrays and takes its workspace from
// one fixed array that lives in this file for as long as the library is
// loaded on a device.  The solve reads its residual back to the host after
// every V-cycle (the stopping rule), so the call synchronises `stream`.
#include <stdio.h>

#include <mutex>

#include "pic_internal.cuh"

namespace {

// Workspace of the solve: FP64 nodal chi and face coefficients of every
// level, coarse right-hand sides and corrections, the fine residual and
// right-hand side.  800,000 doubles (6.4 MB) holds meshes up to 129 x 513
// nodes.
constexpr size_t kNoallocDoubles = 800000;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];
static __device__ __align__(256) pic::DevScalars g_noalloc_scalars;

struct DeviceSlots {
    bool ready = false;
    double *scratch = nullptr;
    pic::DevScalars *scalars = nullptr;
};

constexpr int kMaxDevices = 64;
std::mutex g_mu;
DeviceSlots g_slots[kMaxDevices];

// The symbols above are host-side stand-ins in host code; the device
// addresses are looked up once per device, with that device current, and
// kept for the life of the process.  The cache does not survive a device
// reset (cudaDeviceReset or any other teardown of the device's primary
// context): after one, the addresses it holds are stale.
pic_status device_addresses(double **scratch, pic::DevScalars **scalars) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PIC_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceSlots &s = g_slots[dev];
    if (!s.ready) {
        void *p = nullptr, *q = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return PIC_ERR_CUDA;
        if (cudaGetSymbolAddress(&q, g_noalloc_scalars) != cudaSuccess) return PIC_ERR_CUDA;
        s.scratch = static_cast<double *>(p);
        s.scalars = static_cast<pic::DevScalars *>(q);
        s.ready = true;
    }
    *scratch = s.scratch;
    *scalars = s.scalars;
    return PIC_OK;
}

bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

}  // namespace

extern "C" pic_status pic_field_solve_noalloc(double R, double L, int32_t nz, int32_t nr,
                                              int32_t chi_face, const double *rho,
                                              const double *chi, double V, const double *phi_zL,
                                              double *phi, double tol, int32_t max_cycles,
                                              void *stream, pic_solve_info *info) {
    if (!(R > 0) || !(L > 0) || nz < 3 || !pow2(nz - 1) || nr < 3 || nr > 2049 ||
        (chi_face != PIC_CHI_MAX && chi_face != PIC_CHI_MEAN) || max_cycles < 1 || !rho || !chi ||
        !phi) {
        fprintf(stderr, "pic_field_solve_noalloc: invalid argument\n");
        return PIC_ERR_ARG;
    }
    // carve the workspace: level 0 needs chi and the face coefficients,
    // coarser levels also a right-hand side and a correction
    size_t need = 2 * (size_t)nz * nr;  // fine residual and right-hand side
    int nlev = 0;
    for (int n = nz;; n = (n + 1) / 2) {
        need += (size_t)(nlev == 0 ? 3 : 5) * n * nr;
        ++nlev;
        if (n == 3) break;
    }
    if (need > kNoallocDoubles) {
        fprintf(stderr,
                "pic_field_solve_noalloc: a %d x %d mesh needs %zu doubles of workspace; the "
                "fixed workspace holds %zu (meshes up to 129 x 513)\n",
                nz, nr, need, kNoallocDoubles);
        return PIC_ERR_ARG;
    }
    double *base = nullptr;
    pic::DevScalars *ds = nullptr;
    if (device_addresses(&base, &ds) != PIC_OK) {
        fprintf(stderr, "pic_field_solve_noalloc: cannot resolve the workspace address\n");
        return PIC_ERR_CUDA;
    }
    pic::MGWork mg;
    double *p = base;
    const size_t ng = (size_t)nz * nr;
    mg.r = p;
    p += ng;
    mg.f0 = p;
    p += ng;
    int l = 0;
    for (int n = nz;; n = (n + 1) / 2, ++l) {
        pic::MGLevel &lv = mg.lv[l];
        const size_t g = (size_t)n * nr;
        lv.nz = n;
        lv.dz = L / (n - 1);
        lv.chi = p;
        p += g;
        lv.cz = p;
        p += g;
        lv.cr = p;
        p += g;
        if (l > 0) {
            lv.u = p;
            p += g;
            lv.f = p;
            p += g;
        } else {
            lv.u = nullptr;
            lv.f = nullptr;
        }
        lv.cz32 = lv.cr32 = lv.u32 = lv.f32 = nullptr;
        if (n == 3) break;
    }
    mg.nlev = nlev;
    mg.ds = ds;
    pic::FieldDims fd{nz, nr, L / (nz - 1), R / (nr - 1), L, chi_face};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int launches = 0;
    double res = 0.0;
    const int r = pic::mg_solve(fd, mg, rho, chi, V, phi_zL, phi, false, false, tol, max_cycles,
                                &res, &launches, st);
    if (cudaGetLastError() != cudaSuccess) return PIC_ERR_CUDA;
    if (info) {
        info->cycles = r >= 0 ? r : -r - 1;
        info->rel_residual = res;
    }
    return r >= 0 ? PIC_OK : PIC_ERR_NOT_CONVERGED;
}
