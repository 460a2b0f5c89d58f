"""The residual R(U) as a torch.autograd.Function over the C ABI.

forward      R = sdrt_residual(U)
backward     dL/dU = sdrt_vjp(U, dL/dR)       (reverse mode)
jvp          dR = sdrt_jvp(U, dU)              (forward mode)

U is a flat CUDA state array in the mesh's layout (Mesh.pack); the padding
entries of R and of the products are zero."""
import torch


class Residual(torch.autograd.Function):
    @staticmethod
    def forward(U, mesh):
        R = torch.zeros_like(U)
        mesh.residual(U, R)
        return R

    @staticmethod
    def setup_context(ctx, inputs, output):
        U, mesh = inputs
        ctx.mesh = mesh
        ctx.save_for_backward(U)
        ctx.save_for_forward(U)

    @staticmethod
    def backward(ctx, gR):
        (U,) = ctx.saved_tensors
        out = torch.zeros_like(U)
        ctx.mesh.vjp(U, gR.contiguous(), out)
        return out, None

    @staticmethod
    def jvp(ctx, dU, _mesh_tangent):
        (U,) = ctx.saved_tensors
        out = torch.zeros_like(U)
        ctx.mesh.jvp(U, dU.contiguous(), out)
        return out


def residual(U, mesh):
    """R(U) for a Mesh, differentiable in both modes."""
    return Residual.apply(U, mesh)
