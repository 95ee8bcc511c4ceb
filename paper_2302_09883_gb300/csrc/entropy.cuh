// Lossless entropy stage over the records of a compressed state (order-0
// byte-wise rANS; the layout and the coder are described in entropy.cu).
#pragma once
#include <cuda_runtime.h>

#include <vector>

namespace wcs {
// Codes the npatch records at arena (table tab: offset << 24 | bytes) into
// out (host), decodes them again on the device and sets *mismatches to the
// number of bytes that did not come back.  Synchronises the stream.
cudaError_t entropy_code_state(const unsigned char* arena, const unsigned long long* tab, int npatch,
                               cudaStream_t stream, std::vector<unsigned char>& out, unsigned long long* mismatches);
}  // namespace wcs
