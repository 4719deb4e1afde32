"""Parareal with the time slices sharded over ranks (one process per GPU).

The parallel loop over slices of the parareal iteration (Sec. 3, Eq. 3.1,
Algorithm 4) splits into contiguous blocks, one per rank: rank r owns slices
[a_r, b_r) (`block_bounds`).  One iteration k -> k+1 on rank r:

  1. F and G of the previous iterate on its own slices (the parallel work),
     and V_n = F(U_n^k) - G(U_n^k) for n in [a_r, b_r);
  2. the serial chain over its own links, U_{n+1}^{k+1} = G(U_n^{k+1}) + V_n,
     started from U_{a_r}^{k+1}, which rank r-1 sends when its own segment is
     done (rank 0 starts from u0), and ending with U_{b_r}^{k+1} sent on to rank
     r+1 -- the one exchange of the iteration, a point-to-point hand-off of a
     single state at each block boundary;
  3. the largest relative change over all slices (one max all-reduce of a scalar).

A rank keeps only the states of its own block (and the boundary state it
receives).  The predictor is the same chain with V = 0.  The arithmetic per
slice and per link is that of the single-process iteration, so the iterates
are those of the unsharded method; only where each slice is computed changes.

F and G are callables on a batch of states, torch tensors of shape
(batch, 3, N/2+1) complex128 on the rank's device: `context_propagators` makes
them from a C-ABI context (arp_fine_batch, arp_coarse_step) on the rank's GPU;
tests pass CPU functions.  Communication goes through torch.distributed (NCCL
between GPUs; gloo on the CPU), with states sent as their real views.
"""
from __future__ import annotations

from typing import Callable, Optional

import torch
import torch.distributed as dist

Propagator = Callable[[torch.Tensor], torch.Tensor]


def block_bounds(slices: int, world: int) -> list[tuple[int, int]]:
    """Contiguous blocks [a_r, b_r) of slices 0..slices-1, sizes differing by at most one
    (the first slices % world ranks get one more)."""
    if slices < 1 or world < 1:
        raise ValueError("need at least one slice and one rank")
    base, extra = divmod(slices, world)
    out, a = [], 0
    for r in range(world):
        b = a + base + (1 if r < extra else 0)
        out.append((a, b))
        a = b
    return out


def _parseval(x: torch.Tensor) -> torch.Tensor:
    """Per state: the L2 norm over the three fields by Parseval (weight 1 at k = 0, 2 above)."""
    w = torch.full((x.shape[-1],), 2.0, dtype=torch.float64, device=x.device)
    w[0] = 1.0
    return torch.sqrt(torch.sum(w * (x.real ** 2 + x.imag ** 2), dim=(-2, -1)))


class ShardedParareal:
    """The parareal iteration of one problem with its slices spread over the ranks
    of `group` (the default process group when None)."""

    def __init__(self, F: Propagator, G: Propagator, u0: torch.Tensor, slices: int,
                 group: Optional[dist.ProcessGroup] = None):
        self.F, self.G, self.group = F, G, group
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.slices = slices
        self.a, self.b = block_bounds(slices, self.world)[self.rank]
        self.u0 = u0.reshape(1, *u0.shape[-2:])
        self.level = -1
        # U_a .. U_b of this rank's block (its own slices' start states and the end state)
        self.U: Optional[torch.Tensor] = None

    # --- exchange -----------------------------------------------------------
    def _recv_start(self) -> torch.Tensor:
        if self.rank == 0:
            return self.u0.clone()
        buf = torch.empty_like(torch.view_as_real(self.u0))
        dist.recv(buf, src=self._global(self.rank - 1), group=self.group)
        return torch.view_as_complex(buf)

    def _send_end(self, state: torch.Tensor) -> None:
        if self.rank + 1 < self.world:
            dist.send(torch.view_as_real(state.contiguous()), dst=self._global(self.rank + 1), group=self.group)

    def _global(self, r: int) -> int:
        return dist.get_global_rank(self.group, r) if self.group is not None else r

    def _max_over_ranks(self, x: float) -> float:
        if self.world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=self.u0.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=self.group)
        return float(t.item())

    # --- the iteration --------------------------------------------------------
    def _chain(self, V: Optional[torch.Tensor]) -> torch.Tensor:
        """The serial links of this block: U_{n+1} = G(U_n) (+ V_n), n = a..b-1."""
        n_own = self.b - self.a
        out = torch.empty((n_own + 1,) + tuple(self.u0.shape[1:]), dtype=self.u0.dtype, device=self.u0.device)
        out[0:1] = self._recv_start()
        for i in range(n_own):
            g = self.G(out[i:i + 1])
            out[i + 1:i + 2] = g if V is None else g + V[i:i + 1]
        self._send_end(out[n_own:n_own + 1])
        return out

    def iterate(self) -> tuple[int, float]:
        """One level: the predictor on the first call, then parareal iterations.
        Returns (level, max relative change over all slices; inf for the predictor)."""
        if self.level < 0:
            self.U = self._chain(None)
            self.level = 0
            return self.level, float("inf")
        own = self.U[:-1]
        V = self.F(own) - self.G(own)
        new = self._chain(V)
        d = _parseval(new[1:] - self.U[1:])
        n = _parseval(new[1:])
        local = float(torch.max(d / torch.where(n > 0, n, torch.ones_like(n)))) if len(n) else 0.0
        self.U = new
        self.level += 1
        return self.level, self._max_over_ranks(local)

    def gather(self) -> Optional[torch.Tensor]:
        """All slices U_0..U_S on rank 0 (None elsewhere): for checking and output."""
        own = self.U[1:] if self.rank > 0 else self.U
        if self.world == 1:
            return own.clone()
        sizes = [b - a + (1 if r == 0 else 0) for r, (a, b) in enumerate(block_bounds(self.slices, self.world))]
        if self.rank == 0:
            parts = [torch.view_as_real(own.contiguous())]
            for r in range(1, self.world):
                buf = torch.empty((sizes[r],) + tuple(parts[0].shape[1:]), dtype=torch.float64, device=own.device)
                dist.recv(buf, src=self._global(r), group=self.group)
                parts.append(buf)
            return torch.view_as_complex(torch.cat(parts).contiguous())
        dist.send(torch.view_as_real(own.contiguous()), dst=self._global(0), group=self.group)
        return None


def context_propagators(solver, stream=None) -> tuple[Propagator, Propagator]:
    """F and G of a C-ABI context (binding.Solver) on this rank's GPU: the fine
    sweep (arp_fine_batch) and the coarse step (arp_coarse_step) of a batch of
    device states."""
    from . import binding as b

    def F(x: torch.Tensor) -> torch.Tensor:
        out = torch.empty_like(x)
        b.arp_fine_batch(solver.ctx, x.contiguous(), out, stream)
        return out

    def G(x: torch.Tensor) -> torch.Tensor:
        out = torch.empty_like(x)
        b.arp_coarse_step(solver.ctx, x.contiguous(), out, stream)
        return out

    return F, G
