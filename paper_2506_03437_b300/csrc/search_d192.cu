// The search kernel for d = 192 (8 lanes per row, 6 float4 of the query per lane).
#include "search_impl.cuh"

namespace qk {
template qk_status launch_one<8, 6>(const SearchArgs& a, cudaStream_t stream);
}  // namespace qk
