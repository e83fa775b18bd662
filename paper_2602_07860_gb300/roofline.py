"""Algorithmic work model of the raster kernels (FP32 CUDA-core bound; no tensor-core work).

Units (counted by ``Context.count_candidates`` and from the workload sizes):
  N_cand   (pixel, sub-frame, triangle) triples whose triangle's bounding box at that sub-frame,
           dilated by sqrt(delta ln 1e12), contains the pixel centre -- the "barycentric weights
           for every pixel w.r.t. the relevant triangles, for every frame" of Sec. 3.1.
  N_sample H * W * T pixel x sub-frame samples.

Per-unit flops (an FMA counts 2), fixed once from the formulas, not from compiled code:
  FLOPS_PER_CAND = 12   barycentric solve + coverage of one triple with the per-(triangle, frame)
                        part of adj(F) hoisted: three edge functions a u + b v + c, 2 FMA each.
  FLOPS_PER_SAMPLE = 60 shading of the sample's winner: w = N / D (1 div + 3 mul), albedo and
                        normal interpolation (18 FMA), normalisation (3 FMA + rsqrt + 3 mul),
                        n.l (3 FMA), Lambert and accumulation (~8).
  FLOPS_PER_SAMPLE_BWD = 110  adjoint of the shading (~70) and of w = N / D through the edge
                        functions to the vertex positions (~40).
The soft-coverage term (about 45 flops + exp per uncovered triple within the soft radius) is not
counted, so the model is a lower bound of the useful work.

Peak: 152 SMs x 128 FP32 lanes x 2 flops x 2.070 GHz (maximum SM clock) = 80.6 TFLOP/s.
"""

FLOPS_PER_CAND = 12
FLOPS_PER_SAMPLE = 60
FLOPS_PER_SAMPLE_BWD = 110
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


def fwd_flops(n_cand, n_sample):
    return FLOPS_PER_CAND * n_cand + FLOPS_PER_SAMPLE * n_sample


def bwd_flops(n_cand, n_sample):
    # the adjoint recomputes coverage and shading, then back-propagates per sample
    return FLOPS_PER_CAND * n_cand + (FLOPS_PER_SAMPLE + FLOPS_PER_SAMPLE_BWD) * n_sample


def fp32_peak_tflops(num_sms, mhz=SM_MAX_MHZ):
    return num_sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
