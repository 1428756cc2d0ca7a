"""The algorithmic work and bytes per frame that bench.py divides by
(roofline `achieved`): (K+1) operator applications per Newton step, per
channel (4N + 2G + 2Gc) pruned length-G transforms at 5 G log2 G flops plus
the pointwise products; per CG iteration 10 n_x vector accesses, the coil
maps, rho and the real PSF (CPU only)."""
import bench


def test_work_and_bytes_by_hand_for_one_small_case():
    """N=8, G=16, Gc=4, J=2, one Newton step of one CG iteration: two
    operator applications, each per channel (32 + 32 + 8) transforms of 16
    points at 5*16*4 flops + 28*64 + 2*256 + 4*16 pointwise; per iteration
    8 bytes x (10 n_x + J N^2 + N^2) + 4 G^2 with n_x = 64 + 2*16."""
    per_ch = 72 * 320 + 1792 + 512 + 64
    assert bench.flops_per_frame(8, 16, 4, 2, 1, 1) == 2 * 2 * per_ch
    nx = 64 + 2 * 16
    assert bench.bytes_per_frame(8, 16, 4, 2, 1, 1) == 2 * (8 * (10 * nx + 2 * 64 + 64) + 4 * 256)


def test_work_scales_with_channels_and_iterations():
    """Linear in the channel count and in M (K + 1); the stream size's frame
    is 77 applications of about 201 MFLOP and 9.8 MB per CG iteration."""
    f1 = bench.flops_per_frame(160, 320, 80, 10, 7, 10)
    assert bench.flops_per_frame(160, 320, 80, 20, 7, 10) == 2 * f1
    assert abs(bench.flops_per_frame(160, 320, 80, 10, 14, 10) - 2 * f1) < 1e-6 * f1
    assert abs(f1 / 77 / 1e6 - 201.2) < 0.1
    b1 = bench.bytes_per_frame(160, 320, 80, 10, 7, 10)
    assert abs(b1 / 77 / 1e6 - 9.83) < 0.01
