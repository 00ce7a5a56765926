"""torch.autograd.Function over the library's mobility solve and its
hand-written adjoint (rbfib_mobility_solve / rbfib_mobility_solve_adjoint).

    U = MobilitySolve.apply(r, slip, grid, FT)

r: blob positions (N_bl*3, FP64, CUDA, independent inputs); slip: active slip
(N_bl*3); grid: a binding.Grid with the bodies set; FT: forces/torques
(N_b*6).  The forward solution is kept as the checkpoint for the backward,
which runs one adjoint solve and the kernel-derivative terms on the GPU.
"""
import torch


class MobilitySolve(torch.autograd.Function):
    last_info = {}

    @staticmethod
    def forward(ctx, r, slip, grid, FT):
        grid.set_blob_positions(r.detach().contiguous())
        U, info, x = grid.mobility_solve(FT.detach().contiguous(), slip=slip.detach().contiguous(), return_x=True)
        ctx.grid = grid
        ctx.save_for_backward(x)
        ctx.info = info
        MobilitySolve.last_info = info
        return U

    @staticmethod
    def backward(ctx, gU):
        (x,) = ctx.saved_tensors
        dr, dslip, info = ctx.grid.mobility_solve_adjoint(gU.contiguous().double(), x)
        return dr, dslip, None, None
