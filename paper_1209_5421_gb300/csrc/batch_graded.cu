// The batched-solve kernels for batches that hold systems with big aggregates (graded
// meshes): their finest-level Gauss-Seidel colours and restriction take the level-ordered
// big-aggregate phase. A translation unit of its own so that it compiles beside batch.cu.
#include "batch_kernel.cuh"

namespace amg {

void *batch_kernel_graded(bool fp32, int shape) {
    return fp32 ? batch_kernel_of<float, true>(shape) : batch_kernel_of<double, true>(shape);
}

}  // namespace amg
