// The search kernel for d = 1024 (32 lanes per row, 8 float4 of the query per lane).
#include "search_impl.cuh"

namespace qk {
template qk_status launch_one<32, 8>(const SearchArgs& a, cudaStream_t stream);
}  // namespace qk
