"""Helpers of the GPU parity tests: move seeded inputs to the device, call the
library through its binding, bring results back as numpy."""
import numpy as np
import torch

import oracle
from paper_1807_11830_gb300 import build as sense_build
from paper_1807_11830_gb300 import sense

DEV = "cuda:0"
OP_TOL = 1e-5     # relative L2 per operator application (FP32 path vs FP64 oracle)
CG_TOL = 1e-4     # relative L2 of the CG image after a fixed iteration count


def ensure_built():
    sense_build.build()
    sense.load_library()


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def c64(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).to(DEV)


def i32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).to(DEV)


def bf16_pairs_from_oracle(a):
    """complex array -> bf16 [...,2] device tensor, rounded by the oracle's RNE."""
    f32 = np.ascontiguousarray(a, dtype=np.complex64).view(np.float32)
    bits = oracle.bf16_rne(f32).reshape(tuple(np.shape(a)) + (2,))
    return torch.from_numpy(bits.view(np.int16)).to(DEV).view(torch.bfloat16)


def bf16_pairs_to_complex(t):
    bits = t.view(torch.int16).cpu().numpy().view(np.uint16)
    f = oracle.bf16_to_f32(bits)
    return f[..., 0].astype(np.float64) + 1j * f[..., 1].astype(np.float64)


def make_plan(S, lines, storage=sense.STORE_C64):
    C, ny, nx = S.shape
    F, L = lines.shape
    return sense.Plan(ny, nx, C, F, L, storage)


def storage_tensor(a, storage):
    return c64(a) if storage == sense.STORE_C64 else bf16_pairs_from_oracle(a)


def gpu_forward(x, S, lines, storage=sense.STORE_C64):
    F, ny, nx = x.shape
    C, L = S.shape[0], lines.shape[1]
    plan = make_plan(S, lines, storage)
    St = storage_tensor(S, storage)
    if storage == sense.STORE_C64:
        y = torch.empty((F, C, L, nx), dtype=torch.complex64, device=DEV)
    else:
        y = torch.empty((F, C, L, nx, 2), dtype=torch.bfloat16, device=DEV)
    sense.sense_forward(plan, c64(x), St, i32(lines), y)
    sense.sense_plan_check(plan)
    if storage == sense.STORE_C64:
        return y.cpu().numpy().astype(np.complex128)
    return bf16_pairs_to_complex(y)


def gpu_adjoint(y, S, lines, storage=sense.STORE_C64):
    F, C, L, nx = y.shape
    ny = S.shape[1]
    plan = make_plan(S, lines, storage)
    x = torch.empty((F, ny, nx), dtype=torch.complex64, device=DEV)
    sense.sense_adjoint(plan, storage_tensor(y, storage), storage_tensor(S, storage), i32(lines), x)
    sense.sense_plan_check(plan)
    return x.cpu().numpy().astype(np.complex128)


def gpu_normal(x, S, lines, storage=sense.STORE_C64):
    plan = make_plan(S, lines, storage)
    out = torch.empty(x.shape, dtype=torch.complex64, device=DEV)
    sense.sense_normal(plan, c64(x), storage_tensor(S, storage), i32(lines), out)
    sense.sense_plan_check(plan)
    return out.cpu().numpy().astype(np.complex128)


def gpu_cg(y, S, lines, iters, tol=0.0, storage=sense.STORE_C64, plan=None):
    F, C, L, nx = y.shape
    ny = S.shape[1]
    plan = plan or make_plan(S, lines, storage)
    x = torch.empty((F, ny, nx), dtype=torch.complex64, device=DEV)
    it = torch.zeros(F, dtype=torch.int32, device=DEV)
    rr = torch.zeros(F, dtype=torch.float64, device=DEV)
    oc = torch.zeros(F, dtype=torch.int32, device=DEV)
    sense.sense_cg_solve(plan, storage_tensor(y, storage), storage_tensor(S, storage), i32(lines), iters, tol,
                         x, it, rr, oc)
    sense.sense_plan_check(plan)
    return (x.cpu().numpy().astype(np.complex128), it.cpu().numpy(), rr.cpu().numpy(), oc.cpu().numpy())


def gpu_rss(y, lines, ny, storage=sense.STORE_C64):
    F, C, L, nx = y.shape
    plan = sense.Plan(ny, nx, C, F, L, storage)
    out = torch.empty((F, ny, nx), dtype=torch.float32, device=DEV)
    sense.sense_rss(plan, storage_tensor(y, storage), i32(lines), out)
    sense.sense_plan_check(plan)
    return out.cpu().numpy().astype(np.float64)
