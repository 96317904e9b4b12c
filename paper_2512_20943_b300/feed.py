"""Double-buffered host-to-device feed of per-step inputs.

Per-frame training with inputs that live on the host (a frame's streamed
update map, the frame's target images) copies them to the device every step.
HostFeed overlaps those copies with the previous step's kernels: step k's
inputs go into device slot k % depth on a copy stream of their own, the
consumer's stream waits for that copy (an event) before it reads the slot, and
the copy into a slot waits until the consumer has finished with the slot's
previous contents.  Each step's result (a loss) is copied back into pinned host
memory on the consumer's stream, and `result(k)` waits for step k alone, so a
caller can read step k - 1's loss while step k runs.

Inputs named in `late` are read only later in a step (the targets, by the
backward): `put` does not make the consumer wait for them, `wait(k, name)` does,
so the start of step k (decode, render) overlaps the copy of its late inputs
as well — which matters for the first step, which no earlier step hides.

    feed = HostFeed({"map": ((7, 768, 768), torch.uint16), "target": ((n,), torch.float32)}, rast.stream,
                    late=("target",))
    for k in range(steps):
        dev = feed.put(k, map=map_pinned[k], target=target_pinned[k])
        state = render(dev["map"])                          # enqueued on rast.stream
        feed.wait(k, "target")
        loss = backward(state, dev["target"])
        feed.done(k, loss)
        if k:
            print(feed.result(k - 1))
    print(feed.result(steps - 1))

Host tensors should be pinned (`Tensor.pin_memory()`), otherwise the copies are
synchronous and nothing overlaps.
"""
from __future__ import annotations

import torch


class HostFeed:
    def __init__(self, spec: dict, stream: torch.cuda.Stream, depth: int = 2, result_numel: int = 1,
                 device: torch.device | None = None, late: tuple = ()):
        if depth < 1:
            raise ValueError("depth must be >= 1")
        if set(late) - set(spec):
            raise KeyError(f"no feed buffer named {sorted(set(late) - set(spec))}")
        self.late = tuple(late)
        self.stream = stream
        self.depth = depth
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.copy_stream = torch.cuda.Stream(device=self.device)
        self.slots = [{name: torch.empty(shape, dtype=dtype, device=self.device) for name, (shape, dtype) in
                       spec.items()} for _ in range(depth)]
        self.ready = [{name: torch.cuda.Event() for name in spec} for _ in range(depth)]  # copies finished
        self.free = [torch.cuda.Event() for _ in range(depth)]   # consumer finished with the slot
        self.results = [torch.empty(result_numel, dtype=torch.float32).pin_memory() for _ in range(depth)]
        self.result_step = [-1] * depth
        self.h2d_bytes = sum(t.numel() * t.element_size() for t in self.slots[0].values())

    def put(self, k: int, **host) -> dict:
        """Enqueue the copies of step k's inputs (the others first, the late
        ones after them) and make the consumer wait for all but the late ones;
        returns the device tensors of its slot."""
        s = k % self.depth
        slot = self.slots[s]
        unknown = set(host) - set(slot)
        if unknown:
            raise KeyError(f"no feed buffer named {sorted(unknown)}")
        for name, t in host.items():
            dst = slot[name]
            if t.numel() != dst.numel() or t.dtype != dst.dtype:
                raise ValueError(f"{name}: expected {dst.numel()} x {dst.dtype}, got {t.numel()} x {t.dtype}")
        order = [n for n in host if n not in self.late] + [n for n in host if n in self.late]
        with torch.cuda.stream(self.copy_stream):
            self.copy_stream.wait_event(self.free[s])  # no-op before the slot's first use
            for name in order:
                slot[name].view(-1).copy_(host[name].reshape(-1), non_blocking=True)
                self.ready[s][name].record(self.copy_stream)
        for name in host:
            if name not in self.late:
                self.stream.wait_event(self.ready[s][name])
        return slot

    def wait(self, k: int, name: str) -> None:
        """Make the consumer's stream wait for step k's copy of input `name`
        (for the late inputs, before the work that reads them)."""
        self.stream.wait_event(self.ready[k % self.depth][name])

    def done(self, k: int, result: torch.Tensor | None = None) -> None:
        """Call after step k's work is enqueued on the consumer's stream: queues
        the read-back of its result and releases its slot."""
        s = k % self.depth
        with torch.cuda.stream(self.stream):
            if result is not None:
                self.results[s].copy_(result.detach().reshape(-1).float(), non_blocking=True)
                self.result_step[s] = k
            self.free[s].record(self.stream)

    def result(self, k: int) -> torch.Tensor:
        """Wait for step k and return its result (host tensor, valid until step k + depth's done())."""
        s = k % self.depth
        if self.result_step[s] != k:
            raise KeyError(f"no result of step {k} in the feed")
        self.free[s].synchronize()
        return self.results[s]
