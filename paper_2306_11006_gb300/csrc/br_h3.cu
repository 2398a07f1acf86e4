// br_h3.cu -- blind-rotation kernel shapes with H = 3 (2H warps per gate); gadget length L = 3.
#include "br_kernel.cuh"

namespace arx {

cudaError_t launch_br_h3(const BrArgs &args, int GT, int L, int grid, cudaStream_t st) {
  if (L == 2) {
    return cudaErrorInvalidValue;
  }
  switch (GT) {
    case 1: return br::launch_shape<3, 1, 3>(args, grid, st);
    case 2: return br::launch_shape<3, 2, 3>(args, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

size_t br_smem_h3(int GT, int L) {
  if (L == 2) {
    return 0;
  }
  switch (GT) {
    case 1: return br::br_smem_bytes<3, 1>();
    case 2: return br::br_smem_bytes<3, 2>();
    default: return 0;
  }
}

int br_occupancy_h3(int GT, int L) {
  if (L == 2) {
    return 0;
  }
  switch (GT) {
    case 1: return br::occupancy_shape<3, 1, 3>();
    case 2: return br::occupancy_shape<3, 2, 3>();
    default: return 0;
  }
}

}  // namespace arx
