// Instantiations of the persistent batch kernel for block shapes of 1024 threads (one translation
// unit per thread count, so that the shapes compile in parallel).
#include "block_dev.cuh"

namespace bp {

const void *batch_kernel_1024_1() { return (const void *)k_batch<1024, 1>; }

}  // namespace bp
