"""torch.autograd.Function wrappers of the library's differentiable pieces.

Argument marshalling only; the forward and backward computations run in
libnas.so (nas_apply ops NAS_OP_BVP, NAS_OP_BVP_VJP, NAS_OP_ENERGY_GRAD).

Parameters of the nuclei are packed as a [M, 4] FP64 tensor of rows
(x, y, z, Z).  Moving the nuclei keeps the (fixed) fine and coarse meshes;
gradients are gradients of the discrete problem on that mesh.

* BVPSolve(params, R, solver): U = H~(params)^-1 R, the N shifted linear
  problems of Algorithm 3 at the solver's current density and mu.  Backward:
  the adjoint A = H~^-1 G (a second batched solve with the symmetric
  operator), then dL/dparams = -sum_q W_q dV_ext/dparams(x_q) sum_c a_c u_c
  (an element-wise contraction at the quadrature points) and dL/dR = A.
* KSEnergy(params, solver): total energy of a converged solve (Algorithm 3
  to tol_scf from the coarse-space initial guess); backward: the
  Hellmann-Feynman gradient int rho dV_ext/dparams + dE_nn/dparams, exact
  for the discrete variational problem on the fixed mesh (the Hartree
  boundary values of the paper's eq. bd depend on rho and are not
  variational; without Hartree the gradient is exact).
"""
import numpy as np
import torch

from . import nas


def _set_nuclei(solver, params):
    p = params.detach().cpu().numpy().astype(np.float64)
    inst = solver.inst
    nas.nas_set_system(solver.h, p[:, :3], p[:, 3], inst.potential, inst.smooth_a, inst.occ)


class BVPSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, R, solver):
        _set_nuclei(solver, params)
        Rn = R.detach().cpu().numpy().astype(np.float64)
        U = np.zeros_like(Rn)
        nas.nas_apply(solver.h, nas.NAS_OP_BVP, Rn, U)
        ctx.solver = solver
        ctx.save_for_backward(params, R)
        return torch.from_numpy(U).to(R.device)

    @staticmethod
    def backward(ctx, G):
        params, R = ctx.saved_tensors
        solver = ctx.solver
        _set_nuclei(solver, params)
        Rn = R.detach().cpu().numpy().astype(np.float64)
        Gn = G.detach().cpu().numpy().astype(np.float64)
        n, N = Rn.shape
        M = params.shape[0]
        out = np.zeros(2 * n * N + 4 * M)
        nas.nas_apply(solver.h, nas.NAS_OP_BVP_VJP, np.concatenate([Rn.ravel(), Gn.ravel()]), out)
        A = out[n * N:2 * n * N].reshape(n, N)
        dp = out[2 * n * N:].reshape(M, 4)
        return (torch.from_numpy(dp).to(params.device), torch.from_numpy(A).to(R.device), None)


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
        rho = solver.get(nas.NAS_Q_RHO_IN)
        g = np.zeros((params.shape[0], 4))
        nas.nas_apply(solver.h, nas.NAS_OP_ENERGY_GRAD, rho, g)
        ctx.save_for_backward(torch.from_numpy(g))
        return torch.tensor(E, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gE):
        (g,) = ctx.saved_tensors
        return gE * g.to(gE.device), None
