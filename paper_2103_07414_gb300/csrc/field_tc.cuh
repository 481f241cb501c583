// Tensor-core (tcgen05) field path: declarations shared with the dispatcher.  The launch
// writes the blend reference row into ref (6 floats) before the GEMM reads it.
#pragma once

#include "common.cuh"

// Frame and canvas of the fused field + mosaic update (see blend.cuh).
struct MosaicArgs {
    const uint8_t *frame;
    int fw, fh, pitch, channels;
    uchar4 *canvas;
    int cpitch4, ox, oy;
};

size_t field_tc_workspace_bytes(int n, int grid_w, int grid_h);
emdq_status field_tc_launch(const float *q, const float *c, const float *src, int n, int gx0,
                            int gy0, int gw, int gh, float alpha, float *ref,
                            float2 *disp, char *ws, size_t ws_bytes, cudaStream_t st,
                            const MosaicArgs *mos = nullptr);
