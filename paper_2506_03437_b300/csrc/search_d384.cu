// The search kernel for d = 384 (32 lanes per row, 3 float4 of the query per lane).
#include "search_impl.cuh"

namespace qk {
template qk_status launch_one<32, 3>(const SearchArgs& a, cudaStream_t stream);
}  // namespace qk
