"""Forward + backward steps fed from host memory, with the copies overlapped.

A caller whose scene and upstream gradients live in host memory (a loss computed on
the CPU, a data loader) pays for two transfers per step: the inputs host -> device
and the results (planes and gradients) device -> host.  ``HostPipeline`` hides them
behind the neighbouring steps' kernels: it keeps two device buffer sets (inputs,
renderer planes, gradients), copies step i + 1's inputs in on one stream and step
i - 1's results out on another while step i's forward and backward (replayed from
CUDA graphs captured per buffer set) run on a third.  Every step still performs all
of its copies; only their overlap with other steps' compute changes.

Host tensors must be pinned (page-locked) for the copies to be asynchronous.  A
step's host outputs are complete when the event ``submit`` returns has completed
(``event.synchronize()``); the caller must not overwrite a step's host inputs
before that step's input event (``last_input_event``) or read its outputs before
its output event.
"""

from __future__ import annotations

import torch

from . import fmb

INPUTS = ("means", "chol", "weights", "poses", "g_depth", "g_alpha", "g_normal", "g_flow")


class HostPipeline:
    """Double-buffered host-fed render steps of one batch layout."""

    def __init__(self, obj_offsets, views, n_poses, params: fmb.FmbParams, h_init: dict, want_pose=True,
                 device="cuda", use_graphs=True):
        """h_init: host (or device) tensors named as in ``INPUTS`` (None for an absent
        upstream plane) giving the sizes, and the values the set-up runs (the graphs
        are captured after one untimed step on them)."""
        self.device = torch.device(device)
        self.want_pose = want_pose
        self.n_poses = int(n_poses)
        f32 = dict(dtype=torch.float32, device=self.device)
        self.slots = []
        for _ in range(2):
            r = fmb.Renderer(obj_offsets, views, n_poses, params, device=self.device)
            d_in = {k: (None if h_init.get(k) is None else
                        h_init[k].reshape(-1).to(device=self.device, dtype=torch.float32).clone()) for k in INPUTS}
            G = d_in["means"].numel() // 3
            grads = dict(means=torch.empty(G, 3, **f32), chol=torch.empty(G, 6, **f32),
                         weights=torch.empty(G, **f32),
                         poses=torch.empty(self.n_poses, 12, **f32) if want_pose else None)
            self.slots.append(dict(r=r, d_in=d_in, grads=grads, graph=None,
                                   ev_in=torch.cuda.Event(), ev_comp=torch.cuda.Event(),
                                   ev_out=torch.cuda.Event(), used=False))
        self.s_in = torch.cuda.Stream(self.device)
        self.s_comp = torch.cuda.Stream(self.device)
        self.s_out = torch.cuda.Stream(self.device)
        self.i = 0
        self.last_input_event = None
        if use_graphs:
            for sl in self.slots:
                self._capture(sl)

    def outputs(self, slot):
        """Device result tensors of a buffer set, in the order ``submit`` copies them."""
        r, g = slot["r"], slot["grads"]
        return {k: v for k, v in (("depth", r.depth), ("alpha", r.alpha), ("normal", r.normal), ("flow", r.flow),
                                  ("grad_means", g["means"]), ("grad_chol", g["chol"]),
                                  ("grad_weights", g["weights"]), ("grad_poses", g["poses"])) if v is not None}

    def host_outputs(self, pin=True) -> dict:
        """Freshly allocated (pinned) host tensors matching ``outputs``."""
        return {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=pin) for k, v in self.outputs(self.slots[0]).items()}

    def _run(self, sl):
        d, r = sl["d_in"], sl["r"]
        r.forward(d["means"], d["chol"], d["weights"], d["poses"])
        r.backward(d["means"], d["chol"], d["weights"], d["poses"], d["g_depth"], d["g_alpha"], d["g_normal"],
                   d["g_flow"], want_pose=self.want_pose, out=sl["grads"])

    def _capture(self, sl):
        # warm-up on a side stream (lazy set-up must not happen during capture), then capture
        side = torch.cuda.Stream(self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            self._run(sl)
        torch.cuda.current_stream(self.device).wait_stream(side)
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._run(sl)
        sl["graph"] = g

    def submit(self, h_in: dict, h_out: dict) -> torch.cuda.Event:
        """Enqueues one step: copy ``h_in`` (host tensors named as in ``INPUTS``) to
        the device, render and differentiate, copy the results into ``h_out`` (from
        ``host_outputs``).  Returns the event after which ``h_out`` holds them."""
        sl = self.slots[self.i % 2]
        self.i += 1
        with torch.cuda.stream(self.s_in):
            if sl["used"]:
                self.s_in.wait_event(sl["ev_comp"])  # the slot's previous step has read its inputs
            for k, d in sl["d_in"].items():
                if d is not None:
                    d.copy_(h_in[k].reshape(-1), non_blocking=True)
            sl["ev_in"].record(self.s_in)
        with torch.cuda.stream(self.s_comp):
            self.s_comp.wait_event(sl["ev_in"])
            if sl["used"]:
                self.s_comp.wait_event(sl["ev_out"])  # the slot's previous results are out
            if sl["graph"] is not None:
                sl["graph"].replay()
            else:
                self._run(sl)
            sl["ev_comp"].record(self.s_comp)
        with torch.cuda.stream(self.s_out):
            self.s_out.wait_event(sl["ev_comp"])
            for k, d in self.outputs(sl).items():
                h_out[k].copy_(d, non_blocking=True)
            sl["ev_out"].record(self.s_out)
        sl["used"] = True
        self.last_input_event = sl["ev_in"]
        return sl["ev_out"]

    def streams(self):
        return self.s_in, self.s_comp, self.s_out

    # ---------------------------------------------------------------- fixed host buffers
    # A caller whose host buffers stay the same from step to step (a pinned staging
    # area that a data loader refills, say) can have each buffer set's copies captured
    # as CUDA graphs: its inputs' copies in as one graph, its results' copies out as
    # another.  A step then costs the host three graph launches (copies in, the render
    # and adjoint, copies out) on the same three streams and with the same ordering as
    # ``submit``, instead of a launch per copy.  Every replay still performs all of its
    # copies.

    def capture_fixed(self, h_in: dict, h_outs: list):
        """Captures, per buffer set j, the copies of ``h_in`` (pinned host tensors
        named as in ``INPUTS``, shared by both sets) into the set's device inputs and
        of its results into ``h_outs[j]`` (from ``host_outputs``).  Afterwards
        ``submit_fixed`` runs the steps, the sets in turn.  The caller refills ``h_in``
        only after the previous step's ``last_input_event`` and reads ``h_outs[j]``
        after the event of a step of set j."""
        if len(h_outs) != len(self.slots):
            raise ValueError(f"one host output set per buffer set ({len(self.slots)}) expected")
        for h in list(h_in.values()) + [v for o in h_outs for v in o.values()]:
            if h is not None and not h.is_pinned():
                raise ValueError("fixed host buffers must be pinned (page-locked)")
        if any(sl["graph"] is None for sl in self.slots):
            raise RuntimeError("capture_fixed needs the pipeline's graphs (use_graphs=True)")
        torch.cuda.synchronize(self.device)
        for sl, h_out in zip(self.slots, h_outs):
            g_in, g_out = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
            with torch.cuda.graph(g_in):
                for k, d in sl["d_in"].items():
                    if d is not None:
                        d.copy_(h_in[k].reshape(-1), non_blocking=True)
            with torch.cuda.graph(g_out):
                for k, d in self.outputs(sl).items():
                    h_out[k].copy_(d, non_blocking=True)
            sl["graph_in"], sl["graph_out"] = g_in, g_out
        self.i_fixed = 0

    def submit_fixed(self) -> torch.cuda.Event:
        """Enqueues the next step on the captured host buffers (the buffer sets in
        turn, ordered as ``submit`` orders them); returns the event after which that
        step's host outputs are complete."""
        j = self.i_fixed % len(self.slots)
        self.i_fixed += 1
        sl = self.slots[j]
        with torch.cuda.stream(self.s_in):
            if sl["used"]:
                self.s_in.wait_event(sl["ev_comp"])  # the slot's previous step has read its inputs
            sl["graph_in"].replay()
            sl["ev_in"].record(self.s_in)
        with torch.cuda.stream(self.s_comp):
            self.s_comp.wait_event(sl["ev_in"])
            if sl["used"]:
                self.s_comp.wait_event(sl["ev_out"])  # the slot's previous results are out
            sl["graph"].replay()
            sl["ev_comp"].record(self.s_comp)
        with torch.cuda.stream(self.s_out):
            self.s_out.wait_event(sl["ev_comp"])
            sl["graph_out"].replay()
            sl["ev_out"].record(self.s_out)
        sl["used"] = True
        self.last_input_event = sl["ev_in"]
        return sl["ev_out"]
