"""COBA E/I network object over the C ABI (Appendix N, Listing S6).

Allocates the network state with PyTorch on the GPU, fills a ``NetDesc`` and
drives ``bp_network_*`` / ``bp_simulate``.  All per-step work runs in libbp.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


def _require_cuda(device):
    """The library reads every state and matrix pointer as device memory."""
    if torch.device(device).type != "cuda":
        raise ValueError("the network state must live on a CUDA device, got %r" % (device,))


def _check_csr(csr, n):
    """A stored matrix passed to CobaNetwork: CUDA tensors of the types and
    lengths the library reads (a host pointer or a short buffer would be read
    out of bounds on the device)."""
    indptr, indices, data = csr
    for name, t, dt in (("indptr", indptr, torch.int64), ("indices", indices, torch.int32)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous() or t.dtype != dt:
            raise ValueError("csr %s must be a contiguous CUDA %s tensor" % (name, dt))
    if indptr.numel() != n + 1:
        raise ValueError("csr indptr has %d entries, expected n + 1 = %d" % (indptr.numel(), n + 1))
    if data is not None:
        if (not isinstance(data, torch.Tensor) or not data.is_cuda or not data.is_contiguous()
                or data.dtype not in (torch.float32, torch.bfloat16)):
            raise ValueError("csr data must be None or a contiguous CUDA float32 / bfloat16 tensor")
        if data.numel() != indices.numel():
            raise ValueError("csr data and indices differ in length (%d, %d)" % (data.numel(), indices.numel()))


def materialize_network_csr(seed, p, n, n_e, data_dtype=None, device="cuda"):
    """Stored-CSR form of the network's JIT connectivity: rows [0, n_e) are the
    excitatory projection's rows, rows [n_e, n) the inhibitory ones (row
    i - n_e of that projection); identical to what the JIT path regenerates."""
    de = B.bp_jit_desc_init(B.bp_projection_seed(seed, 0), p)
    di = B.bp_jit_desc_init(B.bp_projection_seed(seed, 1), p)
    ipe, ixe, _ = B.jit_materialize(de, n_e, n, device=device)
    ipi, ixi, _ = B.jit_materialize(di, n - n_e, n, device=device)
    indptr = torch.cat([ipe, ipi[1:] + ipe[-1]])
    indices = torch.cat([ixe, ixi])
    data = None
    if data_dtype is not None:
        # equal weights stored per synapse: w_e on E rows, w_i on I rows
        data = torch.empty(indices.numel(), dtype=data_dtype, device=device)
        data[: ixe.numel()] = 0.6
        data[ixe.numel():] = 6.7
    return indptr, indices, data


class CobaNetwork:
    """E/I COBA network of n LIF neurons (first n_e excitatory).

    conn="jit": connectivity regenerated every step from `seed` with
    probability p (default 80/n).  conn="csr": a stored CSR (indptr, indices,
    data) over all n presynaptic rows; data None means homogeneous weights
    w_e / w_i with exact integer event counts.  delay_e / delay_i: synaptic
    delay of the E / I projection in steps (0: spikes act at the next step).
    align="pre": the AlignPre form (one trace per presynaptic neuron, the
    conductances recomputed through the connection matrix every step) instead
    of the merged postsynaptic conductances of AlignPost.
    """

    def __init__(self, n, n_e=None, conn="jit", seed=2024, p=None, V0=None, csr=None, tile_cols=0,
                 params=None, keep_spk=False, keep_spikes=False, delay_e=0, delay_i=0, align="post",
                 device="cuda"):
        _require_cuda(device)
        self.n = int(n)
        if conn == "csr" and csr is not None:
            _check_csr(csr, self.n)
        if V0 is not None and np.asarray(V0).shape != (self.n,):
            raise ValueError("V0 must hold n = %d potentials" % self.n)
        self.n_e = int(n_e if n_e is not None else (4 * self.n) // 5)
        self.p = float(p if p is not None else 80.0 / self.n)
        self.seed = int(seed)
        self.device = device
        self.params = params if params is not None else B.bp_coba_params_default()
        f32, i32 = torch.float32, torch.int32
        if V0 is None:
            V0 = np.full(self.n, -60.0, np.float32)
        self.V = torch.as_tensor(np.asarray(V0, np.float32), device=device).contiguous()
        self.ge = torch.zeros(self.n, dtype=f32, device=device)
        self.gi = torch.zeros(self.n, dtype=f32, device=device)
        self.ref = torch.zeros(self.n, dtype=torch.uint8, device=device)
        self.spike_list = torch.zeros(self.n, dtype=i32, device=device) if keep_spikes else None
        self.n_spikes = torch.zeros(2, dtype=i32, device=device)
        self.totals = torch.zeros(4, dtype=torch.int64, device=device)
        if align not in ("post", "pre"):
            raise ValueError("align must be 'post' or 'pre'")
        self.align = align
        keep_spk = keep_spk or align == "pre"  # the AlignPre trace update reads the flags
        self.spk = torch.zeros(self.n, dtype=torch.uint8, device=device) if keep_spk else None
        self.trace = torch.zeros(self.n, dtype=f32, device=device) if align == "pre" else None
        self.tile_ptr = None
        desc = B.NetDesc()
        desc.n, desc.n_e = self.n, self.n_e
        desc.coba = self.params
        if conn == "jit":
            desc.conn_kind = B.BP_CONN_JIT
            desc.seed = self.seed & (2**64 - 1)
            desc.p = self.p
            counts = True
        elif conn == "csr":
            if csr is None:
                csr = materialize_network_csr(self.seed, self.p, self.n, self.n_e, device=device)
            self.indptr, self.indices, self.data = csr
            desc.conn_kind = B.BP_CONN_CSR
            desc.indptr = self.indptr.data_ptr()
            desc.indices = self.indices.data_ptr()
            desc.data = None if self.data is None else self.data.data_ptr()
            desc.wkind = B._wkind(self.data)
            counts = self.data is None
            if tile_cols:
                size = B.bp_csr_tile_index_size(self.n, self.n, tile_cols)
                self.tile_ptr = torch.empty(size, dtype=i32, device=device)
                B.bp_csr_tile_index(self.indptr, self.indices, self.n, tile_cols, self.tile_ptr)
                desc.tile_ptr = self.tile_ptr.data_ptr()
                desc.tile_cols = tile_cols
        else:
            raise ValueError("conn must be 'jit' or 'csr'")
        ydt = i32 if counts and align == "post" else f32
        # two halves: step t reads half t mod 2 and delivers into the other
        self.ye = torch.zeros(2 * self.n, dtype=ydt, device=device)
        self.yi = torch.zeros(2 * self.n, dtype=ydt, device=device)
        # delayed projections: ring of max(delay) + 2 per-step spike lists
        self.delay_e, self.delay_i = int(delay_e), int(delay_i)
        self.delay_buf = None
        if self.delay_e > 0 or self.delay_i > 0:
            slots = max(self.delay_e, self.delay_i) + 2
            self.delay_buf = torch.zeros(slots * (self.n + 1), dtype=i32, device=device)
        desc.delay_e, desc.delay_i = self.delay_e, self.delay_i
        desc.delay_buf = None if self.delay_buf is None else self.delay_buf.data_ptr()
        desc.align = B.BP_ALIGN_PRE if align == "pre" else B.BP_ALIGN_POST
        desc.trace = None if self.trace is None else self.trace.data_ptr()
        desc.V, desc.ge, desc.gi, desc.ref = (t.data_ptr() for t in (self.V, self.ge, self.gi, self.ref))
        desc.ye, desc.yi = self.ye.data_ptr(), self.yi.data_ptr()
        desc.spike_list = None if self.spike_list is None else self.spike_list.data_ptr()
        desc.n_spikes = self.n_spikes.data_ptr()
        desc.totals = self.totals.data_ptr()
        desc.spk = None if self.spk is None else self.spk.data_ptr()
        self.desc = desc
        self.handle = B.bp_network_create(desc)
        B.bp_network_reset_counters(self.handle)

    def reset_counters(self):
        B.bp_network_reset_counters(self.handle)

    def state_tensors(self):
        """The caller-owned buffers that hold the network's state."""
        names = ("V", "ge", "gi", "ref", "ye", "yi", "n_spikes", "totals", "spk", "spike_list", "delay_buf", "trace")
        return {k: getattr(self, k) for k in names if getattr(self, k, None) is not None}

    def _live_half(self, step):
        """Index (0 / 1) of the accumulator half the next step reads, or None
        when both halves are kept.  Step t reads half t mod 2 and clears it
        while it delivers into the other, so between steps the half that is
        not read next is all zero and a checkpoint needs only the live one
        (AlignPre networks recompute their accumulators every step and keep
        both)."""
        return None if self.align == "pre" else int(step) & 1

    def _checkpoint_views(self, step):
        h = self._live_half(step)
        out = {}
        for k, t in self.state_tensors().items():
            if h is not None and k in ("ye", "yi"):
                t = t[h * self.n:(h + 1) * self.n]
            out[k] = t
        return out

    def checkpoint(self):
        """A copy of the state (device tensors) and the step count: every
        state buffer, the event accumulators as their live half only."""
        step = B.bp_network_step_count(self.handle)
        return {"step": step, "live_half": self._live_half(step),
                "state": {k: t.clone() for k, t in self._checkpoint_views(step).items()}}

    def checkpoint_to_host(self):
        """A checkpoint in pinned host memory (for restoring from the host
        later, e.g. to resume a run in another process).  The live halves of
        the event accumulators are stored as their nonzero words only (index,
        word pairs: between steps they hold the deliveries of the last step's
        spikes, a small share of the neurons)."""
        torch.cuda.synchronize()
        step = B.bp_network_step_count(self.handle)
        views = self._checkpoint_views(step)
        sparse = {}
        if self._live_half(step) is not None:
            for k in ("ye", "yi"):
                x = views.pop(k)
                idx = torch.empty(x.numel(), dtype=torch.int32, device=x.device)
                val = torch.empty(x.numel(), dtype=torch.int32, device=x.device)
                cnt = torch.zeros(1, dtype=torch.int32, device=x.device)
                B.bp_words_compact(x, idx, val, cnt)
                c = int(cnt.item())
                sparse[k] = (idx[:c].to("cpu").pin_memory(), val[:c].to("cpu").pin_memory())
        return {"step": step, "live_half": self._live_half(step), "sparse": sparse,
                "state": {k: t.to("cpu").pin_memory() for k, t in views.items()}}

    def restore(self, ckpt, non_blocking=False):
        """Writes a checkpoint back (into this network or a new one of the
        same configuration) so that the simulation resumes where it was taken:
        the saved buffers are copied in and the other accumulator half is
        zeroed on the device (sparse accumulators: zeroed, then their saved
        words scattered back by bp_words_scatter).  With non_blocking and a pinned host checkpoint
        the copies are enqueued on the current stream without waiting for
        them."""
        h = ckpt.get("live_half")
        if h is not None and h != self._live_half(ckpt["step"]):
            raise ValueError("checkpoint accumulator half does not match its step count")
        sparse = ckpt.get("sparse", {})
        for k, t in self.state_tensors().items():
            if k in sparse:
                # zero, then the saved words into the live half
                idx, val = sparse[k]
                t.zero_()
                di = idx.to(t.device, non_blocking=non_blocking)
                dv = val.to(t.device, non_blocking=non_blocking)
                B.bp_words_scatter(di, dv, idx.numel(), t[h * self.n:(h + 1) * self.n])
            elif h is not None and k in ("ye", "yi"):
                t[h * self.n:(h + 1) * self.n].copy_(ckpt["state"][k], non_blocking=non_blocking)
                t[(1 - h) * self.n:(2 - h) * self.n].zero_()
            else:
                t.copy_(ckpt["state"][k], non_blocking=non_blocking)
        B.bp_network_set_step_count(self.handle, ckpt["step"])

    def state_bytes(self):
        """Bytes of the caller-owned state buffers."""
        return sum(t.numel() * t.element_size() for t in self.state_tensors().values())

    def checkpoint_bytes(self):
        """Bytes a device checkpoint holds (what a restore copies in)."""
        step = B.bp_network_step_count(self.handle)
        return sum(t.numel() * t.element_size() for t in self._checkpoint_views(step).values())

    @staticmethod
    def host_checkpoint_bytes(ckpt):
        """Bytes of a checkpoint_to_host checkpoint (what a restore uploads)."""
        n = sum(t.numel() * t.element_size() for t in ckpt["state"].values())
        return n + sum(a.numel() * a.element_size() + b.numel() * b.element_size()
                       for a, b in ckpt.get("sparse", {}).values())

    def step(self):
        B.bp_network_step(self.handle)

    def simulate(self, T, record=None):
        B.bp_simulate(self.handle, T, record)

    def prepare(self, T):
        """Captures and uploads the CUDA graphs a T-step simulate launches."""
        B.bp_simulate_prepare(self.handle, T)

    def stats(self):
        out = torch.zeros(4, dtype=torch.float64, device=self.device)
        B.bp_network_stats(self.handle, out)
        return out.cpu().numpy()

    def close(self):
        if getattr(self, "handle", None) is not None:
            B.bp_network_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_csr(sizes, seeds, off, p=None, device="cuda"):
    """Stored rows of a batch: each network's JIT connectivity materialised
    (as materialize_network_csr does for one network) and laid out as one CSR
    over the padded concatenated layout, with targets local to each network;
    padding rows are empty."""
    total = int(off[-1])
    lens = torch.zeros(total, dtype=torch.int64, device=device)
    parts = []
    for b, n in enumerate(sizes):
        n = int(n)
        pb = 80.0 / n if p is None else float(p[b])
        ip, ix, _ = materialize_network_csr(int(seeds[b]), pb, n, (4 * n) // 5, device=device)
        lens[int(off[b]):int(off[b]) + n] = ip[1:] - ip[:-1]
        parts.append(ix)
    indptr = torch.zeros(total + 1, dtype=torch.int64, device=device)
    torch.cumsum(lens, 0, out=indptr[1:])
    return indptr, torch.cat(parts)


class BatchedNetworks:
    """Many independent COBA E/I networks (sizes `sizes`, seeds `seeds`,
    connection probability p = 80/n by default) advanced together by the
    batched persistent kernel, with JIT rows (conn="jit") or the same rows
    stored (conn="csr"; `csr` = (indptr, indices) over the padded layout,
    default: batch_csr of the seeds).  State is concatenated; ``view(b)``
    returns network b's slice of a state array."""

    def __init__(self, sizes, seeds, V0=None, p=None, params=None, conn="jit", csr=None, device="cuda"):
        _require_cuda(device)
        sizes = np.ascontiguousarray(sizes, dtype=np.int64)
        if len(seeds) != len(sizes) or (p is not None and len(p) != len(sizes)):
            raise ValueError("sizes, seeds and p must have one entry per network")
        self.sizes = sizes
        self.n_nets = len(sizes)
        self.seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
        self.off = B.bp_batch_layout(sizes)
        total = int(self.off[-1])
        self.device = device
        self.params = params if params is not None else B.bp_coba_params_default()
        f32 = torch.float32
        V = np.full(total, -60.0, np.float32)
        if V0 is not None:
            for b in range(self.n_nets):
                V[self.off[b]:self.off[b] + sizes[b]] = V0[b]
        self.V = torch.as_tensor(V, device=device)
        self.ge = torch.zeros(total, dtype=f32, device=device)
        self.gi = torch.zeros(total, dtype=f32, device=device)
        self.ref = torch.zeros(total, dtype=torch.uint8, device=device)
        self.totals = torch.zeros((self.n_nets, 4), dtype=torch.int64, device=device)
        self._p = None if p is None else np.ascontiguousarray(p, dtype=np.float64)
        d = B.BatchDesc()
        d.n_nets = self.n_nets
        d.n = sizes.ctypes.data
        d.n_e = None
        d.seed = self.seeds.ctypes.data
        d.p = None if self._p is None else self._p.ctypes.data
        d.coba = self.params
        d.V, d.ge, d.gi, d.ref = (t.data_ptr() for t in (self.V, self.ge, self.gi, self.ref))
        d.totals = self.totals.data_ptr()
        if conn not in ("jit", "csr"):
            raise ValueError("conn must be 'jit' or 'csr'")
        self.indptr = self.indices = None
        if conn == "csr":
            if csr is None:
                csr = batch_csr(sizes, self.seeds, self.off, self._p, device=device)
            self.indptr, self.indices = csr
            for name, t, dt in (("indptr", self.indptr, torch.int64), ("indices", self.indices, torch.int32)):
                if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous() or t.dtype != dt:
                    raise ValueError("csr %s must be a contiguous CUDA %s tensor" % (name, dt))
            if self.indptr.numel() != total + 1:
                raise ValueError("csr indptr must have padded_total + 1 = %d entries" % (total + 1))
            if int(self.indptr[-1].item()) > self.indices.numel():
                raise ValueError("csr indices hold fewer entries than indptr[-1]")
            d.indptr, d.indices = self.indptr.data_ptr(), self.indices.data_ptr()
        self.desc = d
        self.handle = B.bp_batch_create(d)

    @staticmethod
    def layout(sizes):
        """Offsets of the padded concatenated layout (numpy int64 [n + 1])."""
        return B.bp_batch_layout(np.ascontiguousarray(sizes, dtype=np.int64))

    def view(self, t, b):
        return t[int(self.off[b]):int(self.off[b]) + int(self.sizes[b])]

    def reset_counters(self):
        B.bp_batch_reset_counters(self.handle)

    def simulate(self, T):
        B.bp_batch_simulate(self.handle, T)

    def prepare(self, T):
        """Captures and uploads the CUDA graph of a T-step simulate."""
        B.bp_batch_prepare(self.handle, T)

    def autotune(self, probe_steps=20):
        return B.bp_batch_autotune(self.handle, probe_steps)

    def tuning(self):
        """(threads, lanes_per_row, ctas_per_sm, stored_rows)."""
        return B.bp_batch_tuning(self.handle)

    def set_tuning(self, threads, lanes_per_row, ctas_per_sm):
        B.bp_batch_set_tuning(self.handle, threads, lanes_per_row, ctas_per_sm)

    def info(self):
        return B.bp_batch_info(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None:
            B.bp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
