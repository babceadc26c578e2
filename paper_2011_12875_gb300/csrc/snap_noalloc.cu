// snap_noalloc.cu -- neighbour-list build that allocates nothing.
//
// Some callers cannot call cudaMalloc.  A host program that hands the GPU's
// memory to its own allocator or pool (an MD engine or a training framework
// that reserves HBM up front) may have no room left outside that pool, and it
// may forbid libraries to take memory the pool counts on.  A caller on a
// latency-critical path cannot afford cudaMalloc either: it may synchronise
// the device and stall work queued on other streams.  For them this file
// offers one entry point that builds the same neighbour list as
// snap_compute's device builder into the caller's output buffers only.  Its
// scratch (an FP32 copy of the positions and a few counters) lives in the
// fixed array below, which every GPU that loads the library holds until the
// process exits.
#include <cmath>
#include <mutex>

#include "snap_gb300.h"
#include "snap_internal.h"

namespace {

constexpr int kNoAllocMaxAtoms = 65536;
constexpr size_t kScratchBytes = sizeof(float4) * kNoAllocMaxAtoms + 256;

// The shared scratch: [0, 16*kNoAllocMaxAtoms) FP32 positions, then 4 ints of
// counters (cleared by every call).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device.  In host code the
// symbol is only a host-side stand-in, so the address has to come from
// cudaGetSymbolAddress, once per device, with that device current.
cudaError_t scratch_address(unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int snap_neighbors_noalloc(int natoms, const double* pos, const double* box,
                                      double rcut, int cap, int* cnt, int* nbr,
                                      signed char* img, double* rij, int* max_count,
                                      void* stream) {
  if (natoms < 0 || natoms > kNoAllocMaxAtoms) return SNAP_ERR_ARG;
  if (cap < 1 || cap > snap::kMaxNeighCap) return SNAP_ERR_ARG;
  if (!(std::isfinite(rcut) && rcut > 0.0)) return SNAP_ERR_ARG;
  if (!box) return SNAP_ERR_BOX;
  // bounded image range (the build's image loop and its signed-byte shifts)
  int S[3];
  if (!snap::image_shifts(box, rcut, S)) return SNAP_ERR_BOX;
  // the set-up (the scratch array's device address) runs on every valid
  // call, also one with no atoms, so a first call with natoms = 0 does it too
  unsigned char* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return SNAP_ERR_CUDA;
  if (natoms == 0) return SNAP_OK;
  if (!pos || !cnt || !nbr || !img || !rij) return SNAP_ERR_ARG;
  float4* pos4 = reinterpret_cast<float4*>(base);
  int* flags = reinterpret_cast<int*>(base + sizeof(float4) * kNoAllocMaxAtoms);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the counters keep the previous call's values: clear them
  if (cudaMemsetAsync(flags, 0, 4 * sizeof(int), s) != cudaSuccess) return SNAP_ERR_CUDA;
  snap::NeighArgs na{};
  na.n = natoms;
  na.K = cap;
  na.pos = pos;
  na.pos4 = pos4;
  na.Lx = box[0];
  na.Ly = box[1];
  na.Lz = box[2];
  na.Sx = S[0];
  na.Sy = S[1];
  na.Sz = S[2];
  na.rcut = rcut;
  na.cnt = cnt;
  na.nbr = nbr;
  na.img = img;
  na.rij = rij;
  na.flags = flags;
  if (snap::launch_pos4(natoms, pos, pos4, s) != cudaSuccess) return SNAP_ERR_CUDA;
  if (snap::launch_neigh_build(na, s) != cudaSuccess) return SNAP_ERR_CUDA;
  if (max_count &&
      cudaMemcpyAsync(max_count, flags, sizeof(int), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return SNAP_ERR_CUDA;
  return SNAP_OK;
}
