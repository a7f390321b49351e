"""The work counts bench.py divides by kernel times (the roofline's
`achieved`), pinned to closed forms: recomputed suffix sites of the
connected-configuration engine (Sec. II.C), issued tensor-core flops per
recomputed site, and FMA-pipe flops per site of the GRU cell (App. A)."""
import bench
from paper_2608_18065_b300.inputs import HamSpec, HParams, ModelSpec


class _W:
    def __init__(self, model, ham, ns):
        self.model, self.ham, self.hp = model, ham, HParams(0.1, 1e3, 0.0, ns=ns)


def test_suffix_sites_tfim_and_cluster():
    # TFIM: the X operator at site j changes sigma from j on: N - j sites for
    # j = 0..N-1, so N(N+1)/2 per sample
    for N, ns in [(100, 1024), (7, 3)]:
        w = _W(ModelSpec(1, N, 1, 64), HamSpec("tfim"), ns)
        assert bench.eloc_suffix_sites(w) == ns * N * (N + 1) // 2
    # ZXZ cluster: X at sites 1..N-2, so (N - 1)N/2 - 1 per sample
    for N, ns in [(64, 512), (5, 2)]:
        w = _W(ModelSpec(1, N, 1, 64, cplx=1), HamSpec("cluster_zxz"), ns)
        assert bench.eloc_suffix_sites(w) == ns * ((N - 1) * N // 2 - 1)
    # connectivity that depends on the sample is counted by the library
    assert bench.eloc_suffix_sites(_W(ModelSpec(2, 4, 4, 64), HamSpec("j1j2"), 8)) is None


def test_tensor_core_flops_per_site():
    # three BF16 products (hi.hi, hi.lo, lo.hi) of M = 1 row: gates K = 64,
    # N = 192 (1D); 2D adds the state mix K = 128, N = 64
    assert bench.eloc_tc_site_flops(ModelSpec(1, 100, 1, 64)) == 3 * 2 * 64 * 192
    assert bench.eloc_tc_site_flops(ModelSpec(1, 200, 1, 32)) == 3 * 2 * 64 * 192  # padded
    assert bench.eloc_tc_site_flops(ModelSpec(2, 10, 10, 64)) == 3 * 2 * (64 * 192 + 128 * 64)
    # streamed engine: [U1; U2] h_{k-1} (K = dh, N = 2dh) and the gates (K = dh, N = 3dh)
    assert bench.eloc_tc_site_flops(ModelSpec(2, 8, 8, 96)) == 3 * 2 * (96 * 192 + 96 * 288)
    assert bench.eloc_tc_site_flops(ModelSpec(2, 8, 8, 128)) == 3 * 2 * (128 * 256 + 128 * 384)


def test_fma_flops_per_site():
    for dh in (8, 32, 64, 128):
        gates = 2 * dh * 3 * dh
        heads = 2 * dh * 2
        assert bench.site_flops(ModelSpec(1, 10, 1, dh)) == gates + heads
        assert bench.site_flops(ModelSpec(1, 10, 1, dh, cplx=1)) == gates + 2 * heads
        assert bench.site_flops(ModelSpec(2, 4, 4, dh, cplx=1)) == gates + 2 * heads + 2 * 2 * dh * dh


def test_engine_selection_matches_the_library():
    # tensor-core E_loc engines: mixed 1D d_h 32 / 64, mixed 2D d_h 64, 96, 128
    used = [(d, dh) for d in (1, 2) for dh in (8, 16, 32, 64, 96, 128)
            if bench.eloc_tc_used(ModelSpec(d, 4, 4 if d == 2 else 1, dh), "mixed")]
    assert used == [(1, 32), (1, 64)] + [(2, dh) for dh in bench.ENGINE2D_DH]
    assert set(bench.ENGINE2D_DH) >= {64, 96, 128}
    assert not bench.eloc_tc_used(ModelSpec(1, 10, 1, 64), "fp64")
