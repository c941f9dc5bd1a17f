"""Batched solves of many independent grids in one CUDA-graph launch.

Every instance of a mixed-size batch is compared with the FP64 oracle (and
so with what it would give alone), across a change of field pointers (a
new graph) and a repeat of the first pointer set (graph replay), including
an in-place instance.
"""

import numpy as np
import pytest

from oracle import ibm_oracle as O
from paper_2406_19920_gb300 import synth
import paper_2406_19920_gb300 as ibm
from tests.gpu_util import TOL_FP32, TOL_FP64, dev, grid, host, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DIMS = [(32, 32, 32), (48, 40, 48), (16, 16, 16), (64, 24, 64), (32, 32, 32), (48, 40, 48), (12, 10, 24),
        (96, 33, 64)]


@pytest.mark.parametrize("prec", [ibm.IBM_FP32_REFINED, ibm.IBM_FP64])
def test_batch_matches_oracle_and_replays(prec):
    dt = torch.float32 if prec == ibm.IBM_FP32_REFINED else torch.float64
    npdt = np.float32 if prec == ibm.IBM_FP32_REFINED else np.float64
    tol = TOL_FP32 if prec == ibm.IBM_FP32_REFINED else TOL_FP64
    grids = [grid(*d) for d in DIMS]
    batch = ibm.ibm_batch_create(DIMS, [g[3:] for g in grids], prec, 1)
    try:
        sets = []
        for rep in range(2):
            rhs, phi, ref = [], [], []
            for i, (d, g) in enumerate(zip(DIMS, grids)):
                b = synth.white_noise(*d, workload=50 + rep, stream=i).astype(npdt).astype(np.float64)
                ref.append(O.poisson_solve(b, g)[0])
                r = dev(b, dt)
                rhs.append(r)
                phi.append(r if i == 3 else torch.empty_like(r))  # instance 3 in place
            sets.append((rhs, phi, ref))
        for rhs, phi, ref in sets + sets[:1]:
            ibm.ibm_batch_poisson(batch, rhs, phi)
            torch.cuda.synchronize()
            for i in range(len(DIMS)):
                err = rel_err(host(phi[i]), ref[i])
                assert err <= tol, (i, DIMS[i], err)
            # refill the in-place instance for the replay
            rhs[3].copy_(dev(O.laplacian(ref[3], grids[3], O.NEUMANN), dt))
    finally:
        ibm.ibm_batch_destroy(batch)


def test_batch_rejects_bad_arguments():
    g = grid(32, 32, 32)
    with pytest.raises(ibm.IbmError):
        ibm.ibm_batch_create([(30, 32, 32)], [g[3:]], ibm.IBM_FP32_REFINED, 1)
