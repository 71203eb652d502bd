"""PyTorch-facing layer: device memory and streams from torch, compute in libpaulirot.

:class:`StateVector` owns a torch complex tensor of 2^n amplitudes on the
current CUDA device and wraps it in a library handle bound to torch's current
stream.  :class:`PauliRotationEnergy` exposes E(theta) = <psi(theta)|H|psi(theta)>
as a ``torch.autograd.Function`` whose backward pass is the library's adjoint
sweep (``rotation_grads``).  Nothing here computes amplitudes itself.
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import torch

from . import capi

_TORCH_DT = {capi.SV_C128: torch.complex128, capi.SV_C64: torch.complex64}


def current_stream_handle() -> int:
    return int(torch.cuda.current_stream().cuda_stream)


class StateVector:
    """An n-qubit state in torch-owned device memory, |0..0> with identity frame."""

    def __init__(self, n_qubits: int, dtype="c128", device=None):
        if not torch.cuda.is_available():
            raise capi.PauliRotError(capi.SV_ECUDA, "StateVector needs a CUDA device")
        self.n = int(n_qubits)
        self.dtype = capi.dtype_code(dtype)
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(dev):
            self.amps = torch.zeros(1 << self.n, dtype=_TORCH_DT[self.dtype], device=dev)
            self.handle = capi.sv_wrap(self.amps.data_ptr(), self.n, self.dtype, current_stream_handle())
        capi.sv_set_basis_state(self.handle, 0)

    # -- lifetime
    def close(self) -> None:
        if getattr(self, "handle", None):
            capi.sv_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bind_current_stream(self) -> None:
        capi.sv_set_stream(self.handle, current_stream_handle())

    # -- C entry points with this handle
    def set_basis_state(self, k: int) -> "StateVector":
        capi.sv_set_basis_state(self.handle, k)
        return self

    def from_host(self, amps: np.ndarray) -> "StateVector":
        capi.sv_from_host(self.handle, amps)
        return self

    def to_host(self, materialize_frame: bool = True) -> np.ndarray:
        return capi.sv_to_host(self.handle, materialize_frame)

    def materialize(self) -> None:
        capi.sv_materialize(self.handle)

    def frame_apply_pauli(self, pauli: str, qubit: int) -> None:
        capi.frame_apply_pauli(self.handle, pauli, qubit)

    def frame(self):
        return capi.frame_get(self.handle)

    def apply_pauli_rotations(self, x, z, angles) -> None:
        capi.apply_pauli_rotations(self.handle, x, z, angles)

    def apply_plan(self, plan: "Plan") -> None:
        capi.plan_apply(self.handle, plan.handle)

    def expval_pauli_sum(self, x, z, coeff):
        return capi.expval_pauli_sum(self.handle, x, z, coeff)

    def copy_from(self, other: "StateVector") -> None:
        capi.sv_copy(self.handle, other.handle)

    # -- checkpoints and tuning
    def save(self, path: str, tag: int = 0) -> None:
        """Write the amplitudes, the Pauli frame and tag to path (sv_save)."""
        capi.sv_save(self.handle, path, tag)

    def load(self, path: str) -> int:
        """Read a checkpoint of the same n and dtype (sv_load); returns its tag."""
        return capi.sv_load(self.handle, path)

    def autotune(self, x, z, angles, max_depth: int = 0, reps: int = 0):
        """Time the list at every fusion depth on this state (overwritten) and
        record the fastest for its size (plan_autotune); returns (depth, ms)."""
        return capi.plan_autotune(self.handle, x, z, angles, max_depth, reps)


class Plan:
    """A rotation list compiled once (fused runs uploaded to the device)."""

    def __init__(self, n_qubits: int, dtype, x, z, angles, fusion_depth: int = -1):
        self.handle = capi.plan_create(n_qubits, dtype, x, z, angles, fusion_depth, current_stream_handle())

    def stats(self):
        return capi.plan_stats(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            capi.plan_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PauliRotationEnergy(torch.autograd.Function):
    """E(theta) = <psi|H|psi>, psi = R_{M-1}(theta_{M-1}) ... R_0(theta_0) psi0.

    forward(theta, psi0, x, z, hx, hz, hc) -> 0-dim float64 tensor; theta is a
    1-D float64 tensor (any device; it is read on the host).  Forward applies
    the rotations to a copy of psi0 (apply_pauli_rotations) and reduces <H>
    (expval_pauli_sum); psi0 is not modified.  Backward runs the library's FP64
    adjoint sweep (rotation_grads) from psi0 for dE/dtheta, so an evaluation
    without a backward pass (e.g. under torch.no_grad) pays for no gradient.
    psi0 must not change between forward and backward.
    """

    @staticmethod
    def forward(ctx, theta, psi0: StateVector, x, z, hx, hz, hc):
        th = theta.detach().to("cpu", torch.float64).numpy().copy()
        dt = "c128" if psi0.dtype == capi.SV_C128 else "c64"
        work = StateVector(psi0.n, dt, device=psi0.amps.device)
        try:
            work.copy_from(psi0)
            work.apply_pauli_rotations(x, z, th)
            e, _ = work.expval_pauli_sum(hx, hz, hc)
        finally:
            work.close()
        ctx.psi0, ctx.args, ctx.theta = psi0, (x, z, hx, hz, hc), th
        return torch.tensor(e, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        x, z, hx, hz, hc = ctx.args
        _, g = capi.rotation_grads(ctx.psi0.handle, x, z, ctx.theta, hx, hz, hc)
        g = torch.from_numpy(g).to(grad_out.device)
        return grad_out * g, None, None, None, None, None, None


def pauli_rotation_energy(theta, psi0: StateVector, x, z, hx, hz, hc):
    return PauliRotationEnergy.apply(theta, psi0, x, z, hx, hz, hc)
