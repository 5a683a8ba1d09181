"""torch.autograd.Function wrappers of the library's differentiable pieces.

Argument marshalling only; the forward and backward computations run in
libnas.so (nas_apply ops NAS_OP_BVP, NAS_OP_BVP_VJP, NAS_OP_ENERGY_GRAD).
CUDA tensors on the solver's device are passed to the library as device
pointers (no host round trip); CPU tensors go through host buffers.

Parameters of the nuclei are packed as a [M, 4] FP64 tensor of rows
(x, y, z, Z).  Moving the nuclei keeps the (fixed) fine and coarse meshes;
gradients are gradients of the discrete problem on that mesh.

* BVPSolve(params, R, solver): U = H~(params)^-1 R, the N shifted linear
  problems of Algorithm 3 at the solver's current density and mu.  Backward:
  the adjoint A = H~^-1 G (a second batched solve with the symmetric
  operator), then dL/dparams = -sum_q W_q dV_ext/dparams(x_q) sum_c a_c u_c
  (an element-wise contraction at the quadrature points) and dL/dR = A.
  The backward needs the H~ of the forward: it raises if any call that
  changes the solver state (a step, a new density, new nuclei, options)
  came between the two.
* KSEnergy(params, solver): total energy of a converged solve (Algorithm 3
  to tol_scf from the coarse-space initial guess); backward: the
  Hellmann-Feynman gradient int rho dV_ext/dparams + dE_nn/dparams, exact
  for the discrete variational problem on the fixed mesh (the Hartree
  boundary values of the paper's Sec. 3.1 (multipole expansion) depend on
  rho and are not variational; without Hartree the gradient is exact).  The
  gradient is computed in the forward, from the converged density, so a
  later change of the solver state does not affect it.
"""
import numpy as np
import torch

from . import nas


def _set_nuclei(solver, params):
    p = params.detach().cpu().numpy().astype(np.float64)
    inst = solver.inst
    nas.nas_set_system(solver.h, p[:, :3], p[:, 3], inst.potential, inst.smooth_a, inst.occ)


def _apply(solver, op, x, out, cnt=0):
    """nas_apply on contiguous FP64 tensors x, out (both CUDA on the solver's
    device, or both CPU).  CUDA tensors: the caller's stream is synchronised
    first (the library works on its own stream and returns after its result
    is in `out`)."""
    if x.is_cuda:
        torch.cuda.current_stream(x.device).synchronize()
        nas.nas_apply(solver.h, op, x.data_ptr(), out.data_ptr(), cnt=cnt or x.numel(), on_device=1)
    else:
        xn = x.numpy()
        on = out.numpy()
        nas.nas_apply(solver.h, op, xn, on, cnt=cnt)


def _device_of(solver, like):
    dev = getattr(solver, "device", 0)
    if like.is_cuda and like.device.index == dev:
        return like.device
    return torch.device("cpu")


class BVPSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, R, solver):
        _set_nuclei(solver, params)
        dev = _device_of(solver, R)
        Rd = R.detach().to(device=dev, dtype=torch.float64).contiguous()
        U = torch.zeros_like(Rd)
        _apply(solver, nas.NAS_OP_BVP, Rd, U)
        ctx.solver = solver
        ctx.state = solver.state_id()
        ctx.save_for_backward(params, R)
        return U.to(R.device)

    @staticmethod
    def backward(ctx, G):
        params, R = ctx.saved_tensors
        solver = ctx.solver
        if solver.state_id() != ctx.state:
            raise RuntimeError("BVPSolve.backward: the solver state changed after the forward "
                               "(a step, a new density, new nuclei or options); H~ of the forward "
                               "is gone, so its adjoint cannot be formed")
        dev = _device_of(solver, R)
        n, N = R.shape
        M = params.shape[0]
        rg = torch.cat([R.detach().to(device=dev, dtype=torch.float64).reshape(-1),
                        G.detach().to(device=dev, dtype=torch.float64).reshape(-1)]).contiguous()
        out = torch.zeros(2 * n * N + 4 * M, dtype=torch.float64, device=dev)
        _apply(solver, nas.NAS_OP_BVP_VJP, rg, out)
        A = out[n * N:2 * n * N].reshape(n, N)
        dp = out[2 * n * N:].reshape(M, 4)
        return dp.to(params.device), A.to(R.device), None


class KSEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, solver):
        _set_nuclei(solver, params)
        solver.init()
        r, rep = nas.nas_solve(solver.h)
        if r != nas.NAS_OK:
            raise nas.NasError(r, "Algorithm 3 did not reach tol_scf within max_outer steps "
                                  "(drho = %.3e)" % rep.drho)
        E = solver.get(nas.NAS_Q_ENERGY)[0]
        dev = _device_of(solver, params)
        sz = solver.sizes()
        rho = torch.empty(sz["ne"] * sz["nq"], dtype=torch.float64, device=dev)
        if rho.is_cuda:
            nas.nas_get(solver.h, nas.NAS_Q_RHO_IN, (rho.data_ptr(), rho.numel() * 8), 1)
        else:
            nas.nas_get(solver.h, nas.NAS_Q_RHO_IN, rho.numpy())
        g = torch.zeros(params.shape[0], 4, dtype=torch.float64, device=dev)
        _apply(solver, nas.NAS_OP_ENERGY_GRAD, rho, g)
        ctx.save_for_backward(g)
        return torch.tensor(E, dtype=torch.float64, device=params.device)

    @staticmethod
    def backward(ctx, gE):
        (g,) = ctx.saved_tensors
        return gE * g.to(gE.device), None
