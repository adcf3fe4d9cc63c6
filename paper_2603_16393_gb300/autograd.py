"""torch.autograd bindings of the likelihood gradient (Sec. 4.2, 5.1).

The paper obtains dJ/dv by automatic differentiation through the wave solver
and the misfit.  Here the two differentiable maps are autograd Functions whose
backward passes are the library's exact discrete adjoints:

  forward_op(v, plan)           d_syn = F(v)       forward: fwi_forward
                                                   backward: fwi_adjoint_grad
  w2_misfit(d_syn, plan, obs)   J = sum W2 / S_obs forward: fwi_w2_misfit
                                                   backward: its adjoint source

so that ``w2_misfit(forward_op(v, plan), plan, obs).sum().backward()`` gives
the same dJ/dv as ``Plan.gradient`` (bitwise: the same kernels run).

Each call of ``forward_op`` keeps its own copy of what the adjoint reads
(the wavefield record, or with ``checkpoint_every = K`` the checkpoints),
allocated from torch's caching allocator and released with the graph, so
several forward calls may be pending before their backward passes.  The
plan's workspace is shared: calls of one plan run in order on the current
stream.  This module only marshals arguments; the chain-rule product of the
adjoint source with the incoming gradient of J is the one scaling done by
torch.
"""
import torch

from . import api


def _stream(device):
    return torch.cuda.current_stream(device)


class _ForwardOp(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, plan):
        v = v.detach().contiguous()
        api._f32(v, plan.model_shape, "v")
        d_syn = torch.empty(plan.data_shape, dtype=torch.float32, device=v.device)
        record = torch.empty(plan.snap_bytes // 4, dtype=torch.float32, device=v.device)
        api.fwi_forward(plan.handle, v, d_syn, record, plan.workspace, _stream(v.device))
        ctx.save_for_backward(v)
        ctx.record = record
        ctx.plan = plan
        return d_syn

    @staticmethod
    def backward(ctx, grad_d):
        (v,) = ctx.saved_tensors
        plan = ctx.plan
        adj = grad_d.detach().to(torch.float32).contiguous()
        grad_v = torch.empty_like(v)
        api.fwi_adjoint_grad(plan.handle, v, adj, ctx.record, grad_v, plan.workspace,
                             _stream(v.device))
        ctx.record = None
        return grad_v, None


class _W2Misfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, d_syn, plan, obs_ctx):
        d_syn = d_syn.detach().contiguous()
        api._f32(d_syn, plan.data_shape, "d_syn")
        B = plan.prob.batch
        J = torch.empty(B, dtype=torch.float32, device=d_syn.device)
        adj = torch.empty(plan.data_shape, dtype=torch.float32, device=d_syn.device) \
            if ctx.needs_input_grad[0] else None
        api.fwi_w2_misfit(plan.handle, obs_ctx, d_syn, J, None, adj, plan.workspace,
                          _stream(d_syn.device))
        ctx.adj = adj
        return J

    @staticmethod
    def backward(ctx, grad_J):
        adj, ctx.adj = ctx.adj, None
        return adj * grad_J.to(adj.dtype).view(-1, 1, 1, 1), None, None


def forward_op(v, plan):
    """d_syn = F(v) for the plan's batch; differentiable in v."""
    return _ForwardOp.apply(v, plan)


def w2_misfit(d_syn, plan, obs_ctx):
    """J [B] of Eq. final_objective against the prepared observations;
    differentiable in d_syn."""
    return _W2Misfit.apply(d_syn, plan, obs_ctx)


def w2_fwi_objective(v, plan, obs_ctx):
    """J(v) [B] = w2_misfit(forward_op(v)); its backward is dJ/dv."""
    return w2_misfit(forward_op(v, plan), plan, obs_ctx)
