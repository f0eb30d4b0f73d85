"""Uneven batching: many instances of different size, coil count, frame count
and acceleration in one persistent launch per size class (GPU).

Each instance's batched result is checked against the FP64 oracle (1e-4 on
the CG image) and against the same instance solved alone by a plan with the
same kernel variant: the two must agree bit for bit, since a frame's
iterates depend only on its own data and its class's variant.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1807_11830_gb300 import sense, synth
from tests.gpu_util import CG_TOL, c64, ensure_built, i32, rel, storage_tensor, bf16_pairs_from_oracle

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


SPECS = [  # n, coils, frames, accel, storage
    dict(n=64, coils=4, frames=2, accel=3, storage=sense.STORE_C64),
    dict(n=128, coils=6, frames=1, accel=2, storage=sense.STORE_C64),
    dict(n=64, coils=3, frames=3, accel=4, storage=sense.STORE_C64),
    dict(n=192, coils=8, frames=2, accel=6, storage=sense.STORE_C64),
    dict(n=128, coils=5, frames=2, accel=4, storage=sense.STORE_BF16),
    dict(n=128, coils=9, frames=1, accel=3, storage=sense.STORE_C64),
]


def _instances(seed0=900):
    out = []
    for k, sp in enumerate(SPECS):
        spec = dict(n=sp["n"], coils=sp["coils"], frames=sp["frames"], accel=sp["accel"],
                    lines=synth.lines_for_acceleration(sp["n"], sp["accel"]), centre=synth.centre_for(sp["n"]))
        p = synth.mix_instance(spec, seed0 + k)
        y = oracle.forward(p.x_true, p.S, p.lines) + p.noise
        out.append((sp["storage"], p, y))
    return out


def _device_io(inst):
    items, keep = [], []
    for storage, p, y in inst:
        F, n = p.x_true.shape[0], p.x_true.shape[1]
        d = dict(y=storage_tensor(y, storage), S=storage_tensor(p.S, storage), lines=i32(p.lines),
                 x_out=torch.empty((F, n, n), dtype=torch.complex64, device=DEV),
                 iters_out=torch.zeros(F, dtype=torch.int32, device=DEV),
                 rel_resid_out=torch.zeros(F, dtype=torch.float64, device=DEV),
                 outcome_out=torch.zeros(F, dtype=torch.int32, device=DEV))
        items.append(d)
    return items


def _shapes(inst):
    return [dict(ny=p.x_true.shape[1], nx=p.x_true.shape[2], coils=p.S.shape[0], frames=p.x_true.shape[0],
                 lines=p.lines.shape[1], storage=storage) for storage, p, _ in inst]


def _q(storage, a):
    return oracle.quantize_c64_bf16(a) if storage == sense.STORE_BF16 else a.astype(np.complex64).astype(np.complex128)


def test_batch_matches_oracle_and_alone():
    K = 8
    inst = _instances()
    batch = sense.Batch(_shapes(inst))
    assert batch.classes == 4  # 64, 128 c64, 128 bf16, 192
    items = _device_io(inst)
    sense.sense_batch_cg_solve(batch, items, K)
    sense.sense_batch_check(batch)
    torch.cuda.synchronize()
    for k, (storage, p, y) in enumerate(inst):
        xb = items[k]["x_out"].cpu().numpy().astype(np.complex128)
        xo, io, _, so = oracle.cg(_q(storage, y), _q(storage, p.S), p.lines, K)
        assert rel(xb, xo) <= CG_TOL, k
        np.testing.assert_array_equal(items[k]["iters_out"].cpu().numpy(), io)
        np.testing.assert_array_equal(items[k]["outcome_out"].cpu().numpy(), so)
        # alone: a plan with the class's default variant, persistent mode
        F, n = p.x_true.shape[0], p.x_true.shape[1]
        plan = sense.Plan(n, n, p.S.shape[0], F, p.lines.shape[1], storage)
        sense.sense_plan_set_cg_mode(plan, sense.CG_MODE_PERSISTENT)
        xa = torch.empty((F, n, n), dtype=torch.complex64, device=DEV)
        sense.sense_cg_solve(plan, items[k]["y"], items[k]["S"], items[k]["lines"], K, 0.0, xa)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(xa.cpu().numpy(), items[k]["x_out"].cpu().numpy())
    # a second solve replays the captured graph and gives the same bits
    first = [d["x_out"].clone() for d in items]
    sense.sense_batch_cg_solve(batch, items, K)
    torch.cuda.synchronize()
    for a, d in zip(first, items):
        assert torch.equal(a, d["x_out"])
    batch.close()


def test_batch_tolerance_and_autotune():
    inst = _instances(seed0=950)[:4]
    batch = sense.Batch(_shapes(inst))
    items = _device_io(inst)
    sense.sense_batch_autotune(batch, items)
    tol = 3e-3
    sense.sense_batch_cg_solve(batch, items, 80, tol)
    sense.sense_batch_check(batch)
    torch.cuda.synchronize()
    for k, (storage, p, y) in enumerate(inst):
        oc = items[k]["outcome_out"].cpu().numpy()
        rr = items[k]["rel_resid_out"].cpu().numpy()
        assert np.all(oc == sense.CG_CONVERGED) and np.all(rr <= tol), k
        xo, io, _, _ = oracle.cg(_q(storage, y), _q(storage, p.S), p.lines, 80, tol)
        it = items[k]["iters_out"].cpu().numpy()
        assert np.all(np.abs(it.astype(int) - io.astype(int)) <= 1), k
    batch.close()
