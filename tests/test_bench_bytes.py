"""The bench's roofline denominators, counted pass by pass (CPU).

The HBM-roofline fraction of the headline divides the compulsory bytes of
one refined 256^3 FP32 solve by its time, so those bytes are pinned here
from the passes themselves: a real field is nx ny nz FP32 values, the half
spectrum ny nz (nx/2 + 1) complex FP32 values; every pass reads its input
and writes its output once.  One refined solve on the slab path is

  forward x rows       read b, write the spectrum
  slab (twice)         read and write the spectrum
  inverse x rows       read the spectrum, write x (the second time also
                       read x, to add the correction to it)
  fused residual pass  read b and x, write the correction's spectrum

and, with the residual as a pass of its own (read b and x, write r), the
correction's forward x rows read r and write its spectrum.
"""

import pytest


def _field(n):
    return 4 * n ** 3


def _spec(n):
    return 8 * n * n * (n // 2 + 1)


@pytest.mark.parametrize("n", [32, 128, 256])
def test_fused_refined_solve_bytes(n):
    import bench
    k = bench.solve_kind_bytes(n, esz=4, refine=1, fused=True)
    F, S = _field(n), _spec(n)
    assert k["forward"] == F + S
    assert k["pencil"] == 2 * (S + S)
    assert k["inverse"] == (S + F) + (S + F + F)
    assert k["residual"] == F + F + S
    assert sum(k.values()) == 6 * F + 8 * S


def test_headline_bytes_at_256():
    import bench
    total = sum(bench.solve_kind_bytes(256).values())
    # six field reads or writes of 64 MiB, eight spectrum reads or writes of
    # 256 * 256 * 129 * 8 B
    assert total == 6 * 67_108_864 + 8 * 67_633_152 == 943_718_400
    # 56.25 B per grid point (the half spectrum is 129/256 of a complex field)
    assert total / 256 ** 3 == 56.25


def test_unfused_refined_solve_bytes():
    import bench
    n = 256
    k = bench.solve_kind_bytes(n, esz=4, refine=1, fused=False)
    F, S = _field(n), _spec(n)
    assert k["forward"] == 2 * (F + S)       # b, then r
    assert k["residual"] == 3 * F            # read b and x, write r
    assert sum(k.values()) == 1_077_936_128  # the fused pass saves r's write and read


def test_unrefined_solve_bytes():
    import bench
    n = 256
    k = bench.solve_kind_bytes(n, esz=4, refine=0)
    F, S = _field(n), _spec(n)
    assert k == {"forward": F + S, "pencil": 2 * S, "inverse": S + F, "residual": 0}


@pytest.mark.parametrize("refine,fused", [(0, True), (1, True), (1, False), (2, False)])
def test_method_bytes_agrees_with_the_per_kind_count(refine, fused):
    """The whole-solve count (the Poisson comparison's denominator) equals
    the per-kind sum (the headline's), and FP64 moves twice the bytes."""
    import bench
    n = 256
    total = sum(bench.solve_kind_bytes(n, esz=4, refine=refine, fused=fused).values())
    assert bench.method_bytes(n, 4, refine, fused=fused) == total
    assert bench.method_bytes(n, 8, refine, fused=fused) == 2 * total
