"""Algorithmic work model of the raster kernels (FP32 CUDA-core bound; no tensor-core work).

Units, counted by the GPU path's own single-precision decisions (``Context.count_work``, pinned
to the oracle's counters by the tests):
  N_box    (pixel, sub-frame, triangle) triples whose triangle's (undilated) bounding box at that
           sub-frame contains the pixel centre: the barycentric solves of Sec. 3.1 that decide
           coverage, which any binned rasteriser has to do.  (N_cand, the same with boxes dilated
           by sqrt(delta ln 1e12), about 20x larger here, is what a solver without binning or
           without the covered/uncovered split evaluates; it is reported, not credited.)
  N_soft   soft-coverage factors 1 - exp(-d/delta) of uncovered samples that can change the
           single-precision product of Eq. back (exp(-d/delta) > 2^-25).
  N_cov    covered samples (shaded by Eq. fore + Lambert).
  N_sample H * W * T pixel x sub-frame samples.

Per-unit flops (an FMA counts 2, a MUFU op 1), fixed once from the formulas, not from compiled
code.  "plain" is the per-sub-frame solve, "fast" the quadratic-rational solver of
Eq. time-dependent2 and the keyframe closest point of Eqs. euc-dist-approx-1..3:
  CAND    coverage test of one N_box triple.  plain: q0 = p - v0 (2), N1, N2 = cross products with
          the hoisted edges (6), N0 = D - N1 - N2 (2), sign tests (2) = 12.  fast: the three
          quadratics N1(tau), N2(tau), D(tau) by Horner from the per-(pixel, segment)
          coefficients (12), N0 (2), sign tests (2) = 16.
  SOFT    one soft factor.  plain: closest point of the triangle by three clamped edge
          projections (3 x 13 = 39), exponent argument, exp, 1 - e, product (4), q0 (2) = 45.
          fast: w(tau) = N / D (Horner 12, rcp + 2 mul 3), p' = F(X) w (6), closest point in
          F(X) (39), F(tau) w* - p with the lerped edges (20), d (3), exp and product (4) = 87.
  COV     shading of a covered sample: w = N / D (4), albedo (18), normal (18), normalisation
          (10), n.l and Lambert (8), accumulation (2) = 60; fast also lerps the three keyframe
          normals to tau (18) = 78.
  SAMPLE  alpha accumulation of any sample (4).
Adjoint (the forward raster stores, per sample, the winner face or the log soft product and the
count of vanishing factors; the adjoint reads them and does not repeat the coverage tests):
  SOFT_BWD  the soft factor recomputed (SOFT: d and the closest point are needed again), the
            exclusive product exp(S - log f) and dA/dd (5), and the derivative of d to the
            vertex coordinates.  plain (Danskin: the closest point moves along the surface):
            g_r = 2 gd r (3), w*_i g_r to three vertices (6) = 9; total 45 + 5 + 9 = 59.
            fast, d = |F(tau) w* - p|^2 with w* the closest point in F(X) of p' = F(X) w(tau):
            g_r (3), w*_i g_r (6), the edge parameter t of w* and its partials to p' and the two
            keyframe-X edge vertices (37), p' = F(X) w to the keyframe-X vertices and to w (23),
            w = N / D quotient rule (11), N = cross products to the vertices at tau, with the
            relative vertices (44), and the keyframe lerp of tau back to the two segment slots
            plus the keyframe-X terms (42) = 166; total 87 + 5 + 166 = 258.
  COV_BWD   recomputed shading (COV) plus its adjoint: I = c shade (8), albedo / colour weights
            (24), Lambert through the normalised normal (22), normal weights and slot normals
            (24 fast, 12 plain), w = N / D (11), relative vertices (26 fast, 6 plain), edge
            functions to the vertices (18), keyframe lerp to the slots (24 fast only) -- adjoint
            fast 157, plain 101; total fast 78 + 157 = 235, plain 60 + 101 = 161.
The z-test of covering candidates and the binning are not counted, so the model is a lower bound
of the arithmetic the method needs.

Peak: 152 SMs x 128 FP32 lanes x 2 flops x 2.070 GHz (maximum SM clock) = 80.6 TFLOP/s.
"""

FLOPS = {
    "plain": dict(cand=12, soft=45, cov=60, sample=4, soft_bwd=59, cov_bwd=161),
    "fast": dict(cand=16, soft=87, cov=78, sample=4, soft_bwd=258, cov_bwd=235),
}
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


def fwd_flops(solver, n_box, n_soft, n_cov, n_sample):
    k = FLOPS[solver]
    return k["cand"] * n_box + k["soft"] * n_soft + k["cov"] * n_cov + k["sample"] * n_sample


def bwd_flops(solver, n_box, n_soft, n_cov, n_sample):
    """n_box is accepted for symmetry with fwd_flops; the adjoint does no coverage tests."""
    k = FLOPS[solver]
    return k["soft_bwd"] * n_soft + k["cov_bwd"] * n_cov + k["sample"] * n_sample


def describe(solver, n_box, n_soft, n_cov, n_sample, backward):
    k = FLOPS[solver]
    s, c = ("soft_bwd", "cov_bwd") if backward else ("soft", "cov")
    box = "" if backward else f"N_box={n_box} x {k['cand']} + "
    return (f"{box}N_soft={n_soft} x {k[s]} + N_cov={n_cov} x {k[c]} + "
            f"N_sample={n_sample} x {k['sample']} flops ({solver} solver)")


def fp32_peak_tflops(num_sms, mhz=SM_MAX_MHZ):
    return num_sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
