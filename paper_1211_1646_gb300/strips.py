"""Spatial decomposition with inactive bands (Sec. 6): one system split into
strips of cell rows, one strip per processor.

The first cell row of every strip makes no trial moves during a sweep's
sub-sweeps, so strips need each other's rows only around the grid shift
(include/hdmc.h, "spatial decomposition").  This module drives strips
through the per-sweep protocol and moves rows between them; all Monte Carlo
work runs in the library (hdmc_strip_* entry points).

    strips = [Strip(N, Lx, Ly, sigma, d, nselect, seed, "fp32", R, k) for k in range(R)]
    run = StripRun(strips, LocalExchange(strips))          # all strips on this GPU
    run.sweep(100); run.sample(); bp, g0 = run.pressure(N, Lx, Ly)

With one strip per rank, DistExchange moves the rows over a
torch.distributed process group (point-to-point send/receive of one row).
StripRun only calls the methods of the strip objects it is given
(subsweeps, shift, get_row, set_halo, sample, histogram, row_buffer), so any
object with those methods can stand in for a library strip.
"""
import numpy as np

from . import hdmc

# rows a strip sends and the halo slot its neighbour stores them in
# (hdmc_strip_get_row / hdmc_strip_set_halo numbering)
LAST_TO_NEXT = [(3, 1, +1)]               # before the shift: row r1-1 -> next strip's halo r0-1
BAND_TO_PREV = [(0, 2, -1)]               # after the shift: band row r0 -> previous strip's halo r1
ALL_HALOS = [(0, 2, -1), (1, 3, -1), (2, 0, +1), (3, 1, +1)]   # before a histogram


class Strip:
    """Strip `strip` of `nstrips` of the system hdmc_create(N, Lx, Ly, sigma,
    d, nselect, seed, precision) would build, on the current CUDA device."""

    def __init__(self, N, Lx, Ly, sigma, d, nselect, seed, precision, nstrips, strip, stream=None, device=None):
        import torch
        self.device = torch.device(device) if device is not None else torch.device("cuda",
                                                                                   torch.cuda.current_device())
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        self.h = None
        self.h = hdmc.hdmc_strip_create(N, Lx, Ly, sigma, d, nselect, seed, precision, nstrips, strip, stream)
        self.strip, self.nstrips = strip, nstrips
        self.r0, self.r1 = hdmc.hdmc_strip_rows(self.h)
        self.row_bytes = hdmc.hdmc_strip_row_bytes(self.h)
        info = hdmc.hdmc_info(self.h)
        self.mx, self.my_local = info["mx"], info["my"]

    def row_buffer(self, host=False):
        import torch
        if host:
            return torch.empty(self.row_bytes, dtype=torch.uint8, pin_memory=True)
        return torch.empty(self.row_bytes, dtype=torch.uint8, device=self.device)

    def subsweeps(self):
        hdmc.hdmc_strip_subsweeps(self.h)

    def shift(self):
        hdmc.hdmc_strip_shift(self.h)

    def get_row(self, which, buf):
        hdmc.hdmc_strip_get_row(self.h, which, buf.data_ptr())

    def set_halo(self, which, buf):
        hdmc.hdmc_strip_set_halo(self.h, which, buf.data_ptr())

    def sample(self):
        hdmc.hdmc_sample(self.h)

    def histogram(self):
        return hdmc.hdmc_strip_histogram(self.h)

    def counters(self):
        return hdmc.hdmc_counters(self.h)

    def own_state(self):
        """(local[rows, mx, 4, 2], counts[rows, mx]) of the strip's own rows r0 .. r1-1."""
        loc, cnt = hdmc.hdmc_get_state(self.h, self.mx * self.my_local)
        rows = self.r1 - self.r0
        loc = loc.reshape(self.my_local, self.mx, 4, 2)[2:2 + rows]
        cnt = cnt.reshape(self.my_local, self.mx)[2:2 + rows]
        return loc, cnt

    def close(self):
        if getattr(self, "h", None) is not None:
            hdmc.hdmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LocalExchange:
    """Every strip lives in this process: rows go from one strip to another
    through a device buffer."""

    def __init__(self, strips):
        self.strips = strips
        self.buf = strips[0].row_buffer()

    def move(self, moves):
        R = len(self.strips)
        for get_which, set_which, step in moves:
            # read every source row before any halo changes: a strip can be
            # its own neighbour (R = 1), or both neighbours of another (R = 2)
            rows = []
            for k, s in enumerate(self.strips):
                b = s.row_buffer()
                s.get_row(get_which, b)
                rows.append(b)
            for k, b in enumerate(rows):
                self.strips[(k + step) % R].set_halo(set_which, b)


class DistExchange:
    """One strip per rank of a torch.distributed process group: each move
    sends a row to the rank `step` away and receives the matching row from
    the rank `step` the other way (point-to-point, no collective on the
    data path).  host=True stages rows in pinned host memory (gloo)."""

    def __init__(self, strip, dist, rank, world, host=False):
        self.s, self.dist, self.rank, self.world = strip, dist, rank, world
        self.sendbuf = strip.row_buffer(host=host)
        self.recvbuf = strip.row_buffer(host=host)

    def move(self, moves):
        for get_which, set_which, step in moves:
            self.s.get_row(get_which, self.sendbuf)
            dst, src = (self.rank + step) % self.world, (self.rank - step) % self.world
            if dst == self.rank:
                self.recvbuf.copy_(self.sendbuf)
            else:
                ops = [self.dist.P2POp(self.dist.isend, self.sendbuf, dst),
                       self.dist.P2POp(self.dist.irecv, self.recvbuf, src)]
                for r in self.dist.batch_isend_irecv(ops):
                    r.wait()
            self.s.set_halo(set_which, self.recvbuf)


class StripRun:
    """The per-sweep protocol of the decomposition over the strips of this
    process (all strips with LocalExchange, one with DistExchange)."""

    def __init__(self, strips, exchange):
        self.strips = list(strips)
        self.ex = exchange

    def sweep(self, n=1):
        for _ in range(n):
            for s in self.strips:
                s.subsweeps()
            self.ex.move(LAST_TO_NEXT)
            for s in self.strips:
                s.shift()
            self.ex.move(BAND_TO_PREV)

    def sample(self):
        self.ex.move(ALL_HALOS)
        for s in self.strips:
            s.sample()

    def histogram(self):
        """Summed contact histogram of this process's strips and the sample count."""
        total, ns = np.zeros(hdmc.HDMC_HIST_BINS, dtype=np.uint64), 0
        for s in self.strips:
            h, ns = s.histogram()
            total += h
        return total, ns

    def pressure(self, N, Lx, Ly, sigma=1.0, dist=None):
        """beta P / rho and g(sigma+) of the whole system (Sec. 4); with a
        process group, the strips' histograms are summed over the ranks."""
        hist, ns = self.histogram()
        if dist is not None:
            import torch
            t = torch.from_numpy(hist.astype(np.int64))
            dist.all_reduce(t)
            hist = t.numpy().astype(np.uint64)
        return hdmc.hdmc_pressure_fit(hist, ns, N, Lx, Ly, sigma)
