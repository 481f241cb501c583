// Tensor-core field path (placeholder until the tcgen05 kernel lands).
#include "field_tc.cuh"

size_t field_tc_workspace_bytes(int, int, int) { return 0; }

emdq_status field_tc_launch(const float *, const float *, const float *, int, int, int, int,
                            int, float, const float *, float2 *, char *, size_t, cudaStream_t)
{
    return EMDQ_ENOTSUP;
}
