"""Differentiable butterfly Legendre stage for PyTorch.

``legendre_synthesis(beta, plan, prec)`` returns G = S beta: the Legendre
synthesis of Section 2 (the sums over k of eq. alternate_expansion) applied
through the butterfly, for one field (beta of shape [T], T = 2l(2l+1)/2) or
a batch of fields (beta of shape [B, T], one launch for the whole batch).

The backward pass is the transposed butterfly without quadrature weights
(Section 2.2, remark after Figure multi): grad_beta = S^T grad_G, through
``sht_legendre_synthesize_adjoint`` (or its batched form).  S is real, so in
PyTorch's convention for complex tensors (grad = dL/dRe + i dL/dIm) the
gradient of the complex-linear map is S^T applied to the complex incoming
gradient, and nothing is saved for the backward pass beyond the plan and
the precision.  Coefficients and G are treated as independent complex
numbers; a loss on the real grid (which counts orders +m and -m) would add
its own factor 2 for m > 0 outside this function.

Batches of fields (beta of shape [B, T]) run as one launch per direction;
the first launch of each direction on a cached batch first runs the batch
autotuner (synchronous, a few launches) to choose how many fields share a
reading of the factor stream.  Make that first call outside any CUDA graph
capture.

Device status: the launches are asynchronous and their bounded waits report
a timeout only in a device status word (the kernel then stops early and its
output is undefined).  Nothing here reads that word unless asked:
``legendre_synthesis(..., check=True)`` synchronizes the stream after the
forward launch and after the backward launch and raises ``sht.ShtError``
on a nonzero status; otherwise call ``device_status(plan, prec, batch)``
(or ``sht.sht_last_device_status``) yourself where it matters.
"""

import torch

from . import sht

_CDT = {sht.SHT_FP64: torch.complex128, sht.SHT_SPLIT32: torch.complex128, sht.SHT_SPLIT32_ACC64: torch.complex128,
        sht.SHT_FP32: torch.complex64}


def _batch(plan, prec, n):
    """Batch of n fields of one plan, cached on the plan object."""
    cache = plan.__dict__.setdefault("_autograd_batches", {})
    key = (int(prec), int(n))
    if key not in cache:
        cache[key] = sht.Batch([plan] * n, prec)
    return cache[key]


def _tune_once(B, direction, ip, op, stream):
    """The batch autotuner (fields per group) on the first launch of each
    direction, with that launch's own pointers (its outputs are overwritten
    by the launch that follows)."""
    done = B.__dict__.setdefault("_tuned", set())
    if direction not in done:
        sht.sht_batch_autotune(B, direction, ip, op, reps=2, stream=stream)
        done.add(direction)


def _apply(plan, prec, x, adjoint):
    l = plan.l
    T = (2 * l) * (2 * l + 1) // 2
    if x.dtype != _CDT[prec]:
        raise TypeError(f"precision {prec} takes {_CDT[prec]}, got {x.dtype}")
    if not x.is_cuda:
        raise ValueError("tensors must be on the GPU")
    x = x.contiguous()
    stream = torch.cuda.current_stream(x.device)
    single = x.dim() == (2 if adjoint else 1)
    xs = x.unsqueeze(0) if single else x
    n = xs.shape[0]
    if tuple(xs.shape[1:]) != ((2 * l, 2 * l) if adjoint else (T,)):
        raise ValueError(f"unexpected shape {tuple(x.shape)} for l={l}")
    out = torch.empty((n, T) if adjoint else (n, 2 * l, 2 * l), dtype=x.dtype, device=x.device)
    if n == 1:
        fn = sht.sht_legendre_synthesize_adjoint if adjoint else sht.sht_legendre_synthesize
        fn(plan, prec, xs[0], out[0], stream)
    else:
        B = _batch(plan, prec, n)
        ip = sht.pointer_array(list(xs), device=x.device)
        op = sht.pointer_array(list(out), device=x.device)
        _tune_once(B, 2 if adjoint else 0, ip, op, stream)  # batch directions: 0 synthesis, 2 its adjoint
        fn = sht.sht_batch_synthesize_adjoint if adjoint else sht.sht_batch_synthesize
        fn(B, ip, op, stream)
        # the pointer arrays must live until the launch has read them
        ip.record_stream(stream)
        op.record_stream(stream)
    return out[0] if single else out


def device_status(plan, prec, nfields=1):
    """Status word of the launches of one field (the plan's) or of a batch of
    nfields fields of this plan (its cached batch); synchronizes the stream.
    0 = fine, 5 = a bounded wait gave up."""
    stream = torch.cuda.current_stream()
    if nfields == 1:
        return sht.sht_last_device_status(plan, stream)
    return sht.sht_batch_last_device_status(_batch(plan, int(prec), nfields), stream)


def _checked(plan, prec, x, n, where):
    code = device_status(plan, prec, n)
    if code != 0:
        raise sht.ShtError(code, where)
    return x


class LegendreSynthesis(torch.autograd.Function):
    """G = S beta with the transposed butterfly as its hand-written backward."""

    @staticmethod
    def forward(ctx, beta, plan, prec, check):
        ctx.plan = plan
        ctx.prec = int(prec)
        ctx.check = bool(check)
        out = _apply(plan, int(prec), beta, adjoint=False)
        n = 1 if beta.dim() == 1 else beta.shape[0]
        return _checked(plan, prec, out, n, "legendre_synthesis forward") if check else out

    @staticmethod
    def backward(ctx, grad_G):
        g = _apply(ctx.plan, ctx.prec, grad_G, adjoint=True)
        if ctx.check:
            g = _checked(ctx.plan, ctx.prec, g, 1 if grad_G.dim() == 2 else grad_G.shape[0],
                         "legendre_synthesis backward")
        return g, None, None, None


def legendre_synthesis(beta, plan, prec=sht.SHT_FP64, check=False):
    """Differentiable Legendre synthesis of one field ([T]) or a batch ([B, T]).
    check=True reads the device status after each launch (synchronizing) and
    raises on a timeout."""
    return LegendreSynthesis.apply(beta, plan, prec, check)
