// br_h2.cu -- blind-rotation kernel shapes with H = 2 (2H warps per gate); gadget length L = 3 and 2.
#include "br_kernel.cuh"

namespace arx {

cudaError_t launch_br_h2(const BrArgs &args, int GT, int L, int grid, cudaStream_t st) {
  if (L == 2) {
    switch (GT) {
      case 1: return br::launch_shape<2, 1, 2>(args, grid, st);
      case 3: return br::launch_shape<2, 3, 2>(args, grid, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (GT) {
    case 1: return br::launch_shape<2, 1, 3>(args, grid, st);
    case 3: return br::launch_shape<2, 3, 3>(args, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

size_t br_smem_h2(int GT, int L) {
  if (L == 2) {
    switch (GT) {
      case 1: return br::br_smem_bytes<2, 1, 2>();
      case 3: return br::br_smem_bytes<2, 3, 2>();
      default: return 0;
    }
  }
  switch (GT) {
    case 1: return br::br_smem_bytes<2, 1>();
    case 3: return br::br_smem_bytes<2, 3>();
    default: return 0;
  }
}

int br_occupancy_h2(int GT, int L) {
  if (L == 2) {
    switch (GT) {
      case 1: return br::occupancy_shape<2, 1, 2>();
      case 3: return br::occupancy_shape<2, 3, 2>();
      default: return 0;
    }
  }
  switch (GT) {
    case 1: return br::occupancy_shape<2, 1, 3>();
    case 3: return br::occupancy_shape<2, 3, 3>();
    default: return 0;
  }
}

}  // namespace arx
