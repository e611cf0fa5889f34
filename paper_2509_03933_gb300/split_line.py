"""Lines split across ranks: the paper's multi-GPU divide and conquer (Section 2.1; Algorithm 2,
Pipelined-v2; Section 3.1, even distribution of Stage B).

Every rank holds a slab of consecutive rows of every line. Per batch of lines:
  Stage A  every rank reduces its slab to two rows per line            (tdma_slab_reduce)
  A2B      all-to-all: the rank that owns a line's Stage B gathers the line's rows from all
           ranks; lines are dealt out in W equal contiguous shares (even distribution)
  Stage B  the 2W-row reduced system of every owned line                (tdma_slab_pairs_solve)
  B2C      all-to-all back: every rank receives its slab's two end values
  Stage C  every rank finishes its slab                                 (tdma_slab_finish)
Batches are pipelined on two CUDA streams: Stage A and Stage C of one batch run on the compute
stream while the exchanges and Stage B of the previous batch run on the second stream, so the
low-occupancy Stage B and the communication hide behind the bandwidth-bound stages.

``SplitLineSolver`` is the schedule and the exchanges (torch.distributed all_to_all_single:
NCCL between GPUs, or any backend whose tensors the stages accept); ``SlabStages`` binds the three
stage kernels of the library. The schedule only moves fixed-size per-line records between ranks,
so other stage implementations with the same record sizes drop in unchanged.
"""
from __future__ import annotations

import contextlib
import ctypes

import torch

from . import TDMAError, _VP, _ptr, _stream, load_library


class SlabDesc(ctypes.Structure):
    _fields_ = [("n_local", ctypes.c_int64), ("n_lines", ctypes.c_int64), ("elem_stride", ctypes.c_int64),
                ("inner_count", ctypes.c_int64), ("inner_stride", ctypes.c_int64),
                ("outer_stride", ctypes.c_int64), ("nrhs", ctypes.c_int32), ("first", ctypes.c_int32),
                ("last", ctypes.c_int32)]


def _bind(lib):
    if getattr(lib, "_slab_bound", False):
        return lib
    st = ctypes.c_int
    lib.tdma_slab_scratch_bytes.argtypes = [ctypes.POINTER(SlabDesc), ctypes.c_int64]
    lib.tdma_slab_scratch_bytes.restype = ctypes.c_size_t
    lib.tdma_slab_pairs_work_bytes.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32]
    lib.tdma_slab_pairs_work_bytes.restype = ctypes.c_size_t
    lib.tdma_slab_reduce.argtypes = [ctypes.POINTER(SlabDesc)] + [_VP] * 4 + [ctypes.c_int64, ctypes.c_int64] + \
        [_VP] * 4
    lib.tdma_slab_reduce.restype = st
    lib.tdma_slab_pairs_solve.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32] + [_VP] * 5
    lib.tdma_slab_pairs_solve.restype = st
    lib.tdma_slab_finish.argtypes = [ctypes.POINTER(SlabDesc), ctypes.c_int64, ctypes.c_int64] + [_VP] * 4
    lib.tdma_slab_finish.restype = st
    lib._slab_bound = True
    return lib


class SlabStages:
    """The three stage kernels for this rank's slab: n_local rows of n_lines lines, addressed as a
    tdma_desc_t (``layout`` = (elem_stride, inner_count, inner_stride, outer_stride)); ``first`` /
    ``last``: the slab holds the lines' first / last rows. FP64; nrhs 1 or 2."""

    def __init__(self, n_local, n_lines, layout, nrhs=1, first=True, last=True, device="cuda"):
        self._lib = _bind(load_library())
        es, ic, isd, osd = layout
        self.desc = SlabDesc(n_local=n_local, n_lines=n_lines, elem_stride=es, inner_count=ic, inner_stride=isd,
                             outer_stride=osd, nrhs=nrhs, first=int(bool(first)), last=int(bool(last)))
        self.nrhs = nrhs
        self.K = 4 + 2 * nrhs      # doubles per line in a reduced record
        self.E = 2 * nrhs          # doubles per line in an end-value record
        self.device = torch.device(device)
        self.status = torch.zeros(4, dtype=torch.int32, device=self.device)

    def scratch(self, count):
        nbytes = self._lib.tdma_slab_scratch_bytes(ctypes.byref(self.desc), count)
        return torch.empty(max(1, nbytes // 8), dtype=torch.float64, device=self.device)

    def work(self, W, count):
        nbytes = self._lib.tdma_slab_pairs_work_bytes(W, count, self.nrhs)
        return torch.empty(max(1, nbytes // 8), dtype=torch.float64, device=self.device)

    def reduce(self, a, b, c, d, line0, count, reduced, scratch, stream=None):
        st = self._lib.tdma_slab_reduce(ctypes.byref(self.desc), _ptr(a), _ptr(b), _ptr(c), _ptr(d), line0, count,
                                        _ptr(reduced), _ptr(scratch), _ptr(self.status), _stream(stream))
        if st != 0:
            raise TDMAError(st, "tdma_slab_reduce")

    def pairs_solve(self, W, count, gathered, ends, work, stream=None):
        st = self._lib.tdma_slab_pairs_solve(W, count, self.nrhs, _ptr(gathered), _ptr(ends), _ptr(work),
                                             _ptr(self.status), _stream(stream))
        if st != 0:
            raise TDMAError(st, "tdma_slab_pairs_solve")

    def finish(self, line0, count, ends, scratch, x, stream=None):
        st = self._lib.tdma_slab_finish(ctypes.byref(self.desc), line0, count, _ptr(ends), _ptr(scratch), _ptr(x),
                                        _stream(stream))
        if st != 0:
            raise TDMAError(st, "tdma_slab_finish")

    def last_error(self):
        """Synchronise and read (and clear) the device status: 0 or TDMA_ERR_NONFINITE."""
        torch.cuda.synchronize(self.device)
        err = int(self.status[0].item())
        self.status.zero_()
        return err


def pipeline_time(n_batches, t_a, t_x, t_c):
    """Modelled time of the schedule of SplitLineSolver for n_batches equal batches whose stages
    take t_a (Stage A), t_x (both exchanges and Stage B) and t_c (Stage C). The compute stream runs
    A_0, A_1, C_0, A_2, C_1, ..., C_{nb-1} in that order; X_k starts when A_k and X_{k-1} are done;
    C_k when X_k is done and the compute stream is free (the paper's pipelined scheduling model,
    Section 4.2.3, for this two-stream form)."""
    ac = xb = 0.0
    x_end = []
    for k in range(n_batches):
        ac += t_a                       # A_k
        xb = max(xb, ac) + t_x          # X_k
        x_end.append(xb)
        if k >= 1:
            ac = max(ac, x_end[k - 1]) + t_c  # C_{k-1}
    if n_batches:
        ac = max(ac, x_end[-1]) + t_c   # C_{nb-1}
    return ac


def choose_batch(n_lines, stage_times):
    """The batch size with the shortest modelled time, from per-batch stage times measured at a few
    batch sizes ({batch: (t_a, t_x, t_c)}): the paper's estimator (Section 4.2.3), which times the
    stages once per candidate instead of solving the whole domain with each."""
    def est(b):
        return pipeline_time(-(-n_lines // b), *stage_times[b])
    return min(stage_times, key=est), {b: est(b) for b in stage_times}


def shares(count, world):
    """Even distribution of a batch's lines over the ranks: contiguous [lo, hi) per rank."""
    return [(count * r // world, count * (r + 1) // world) for r in range(world)]


class SplitLineSolver:
    """Algorithm 2 on this rank: batches of ``batch_lines`` lines, Stage A/C on one stream and the
    exchanges + Stage B on another (two batches in flight), even distribution of Stage B.

    ``stages`` provides reduce / pairs_solve / finish / scratch / work and the record sizes K, E;
    ``group`` is a torch.distributed process group (None: the default group, or a single rank when
    torch.distributed is not initialised). Ranks must be ordered like their slabs along the line."""

    def __init__(self, stages, n_lines, batch_lines, group=None):
        self.stages = stages
        self.n_lines = n_lines
        self.batch = max(1, min(batch_lines, n_lines)) if n_lines > 0 else 1
        dist = torch.distributed
        self.dist = dist if dist.is_available() and dist.is_initialized() else None
        self.group = group
        self.world = self.dist.get_world_size(group) if self.dist else 1
        self.rank = self.dist.get_rank(group) if self.dist else 0
        self.cuda = stages.device.type == "cuda"
        dev = stages.device
        W, K, E, B = self.world, stages.K, stages.E, self.batch
        own_max = max(hi - lo for lo, hi in shares(B, W))
        f64 = dict(dtype=torch.float64, device=dev)
        # two slots: the batch in Stage A/C and the batch in exchange/Stage B
        self.slots = [dict(red=torch.empty(B * K, **f64), gath=torch.empty(W * own_max * K, **f64),
                           ends=torch.empty(W * own_max * E, **f64), back=torch.empty(B * E, **f64),
                           scratch=stages.scratch(B), work=stages.work(W, own_max)) for _ in range(2)]
        if self.cuda:
            self.s_ac = torch.cuda.current_stream(dev)
            self.s_b = torch.cuda.Stream(device=dev)

    def _a2a(self, out, inp, out_splits, in_splits):
        if self.world == 1:
            out[:inp.numel()].copy_(inp)
        else:
            self.dist.all_to_all_single(out, inp, out_splits, in_splits, group=self.group)

    def _ctx(self, s):
        return torch.cuda.stream(s) if self.cuda else contextlib.nullcontext()

    def solve(self, a, b, c, d, x):
        """x = the solution on this rank's slab of every line (a, b, c, d, x: the slab's arrays)."""
        st, W, K, E = self.stages, self.world, self.stages.K, self.stages.E
        batches = [(l0, min(self.batch, self.n_lines - l0)) for l0 in range(0, self.n_lines, self.batch)]
        pending = None  # (line0, count, slot, event) of the batch whose Stage C is due
        for i, (l0, cnt) in enumerate(batches):
            sl = self.slots[i % 2]
            sh = shares(cnt, W)
            lo, hi = sh[self.rank]
            own = hi - lo
            with self._ctx(self.s_ac if self.cuda else None):
                st.reduce(a, b, c, d, l0, cnt, sl["red"], sl["scratch"])
                ev_a = torch.cuda.Event() if self.cuda else None
                if ev_a is not None:
                    ev_a.record()
            with self._ctx(self.s_b if self.cuda else None):
                if ev_a is not None:
                    self.s_b.wait_event(ev_a)
                red = sl["red"][:cnt * K]
                gath = sl["gath"][:W * own * K]
                self._a2a(gath, red, [own * K] * W, [(h - l) * K for l, h in sh])
                ends = sl["ends"][:W * own * E]
                st.pairs_solve(W, own, gath, ends, sl["work"])
                back = sl["back"][:cnt * E]
                self._a2a(back, ends, [(h - l) * E for l, h in sh], [own * E] * W)
                ev_b = torch.cuda.Event() if self.cuda else None
                if ev_b is not None:
                    ev_b.record()
            if pending is not None:
                self._finish(*pending, x)
            pending = (l0, cnt, sl, ev_b)
        if pending is not None:
            self._finish(*pending, x)
        return x

    def measure_stages(self, a, b, c, d, x, reps=3):
        """Per-batch times (t_a, t_x, t_c) of the first batch, each stage timed alone with CUDA
        events (median of ``reps``), the maximum over ranks. All ranks must call this."""
        if not self.cuda:
            raise RuntimeError("stage timing needs CUDA")
        st, W, K, E = self.stages, self.world, self.stages.K, self.stages.E
        cnt = min(self.batch, self.n_lines)
        sl = self.slots[0]
        sh = shares(cnt, W)
        lo, hi = sh[self.rank]
        own = hi - lo
        stream = torch.cuda.current_stream()

        def timed(fn):
            out = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                out.append(e0.elapsed_time(e1))
            return sorted(out)[len(out) // 2]

        def exchange_and_b():
            gath = sl["gath"][:W * own * K]
            self._a2a(gath, sl["red"][:cnt * K], [own * K] * W, [(h - l) * K for l, h in sh])
            ends = sl["ends"][:W * own * E]
            st.pairs_solve(W, own, gath, ends, sl["work"])
            self._a2a(sl["back"][:cnt * E], ends, [(h - l) * E for l, h in sh], [own * E] * W)

        t_a = timed(lambda: st.reduce(a, b, c, d, 0, cnt, sl["red"], sl["scratch"]))
        t_x = timed(exchange_and_b)
        t_c = timed(lambda: st.finish(0, cnt, sl["back"][:cnt * E], sl["scratch"], x))
        t = torch.tensor([t_a, t_x, t_c], dtype=torch.float64, device=self.stages.device)
        if self.world > 1:
            self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return tuple(float(v) for v in t.tolist())

    def _finish(self, l0, cnt, sl, ev, x):
        with self._ctx(self.s_ac if self.cuda else None):
            if ev is not None:
                self.s_ac.wait_event(ev)
            self.stages.finish(l0, cnt, sl["back"][:cnt * self.stages.E], sl["scratch"], x)
