"""Persistent cache of measured kernel timings (JSON), so that a calibration
interrupted part-way resumes without re-timing what it had measured.

The paper caches its symbolic counts between runs; measured times are the
costly part here.  A time is valid only for the device and clock setting it
was taken on, so entries are grouped by a device identity (GPU UUID, name,
the SM clock limits nvidia-smi reports) and keyed by kernel, parameters,
trial count and L2 flush.  Saves are atomic (write a temporary file, then
rename over the cache)."""
import json
import os
import subprocess


def device_identity(torch, dev_index):
    """Identity of CUDA device `dev_index` for cache grouping: UUID, name and
    the SM clock limits (max and application clocks, read-only query)."""
    pr = torch.cuda.get_device_properties(dev_index)
    clocks = None
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(dev_index), "--query-gpu=clocks.max.sm,clocks.applications.graphics",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
        clocks = out.stdout.strip() or None
    except Exception:
        clocks = None
    return {"uuid": str(getattr(pr, "uuid", "")), "name": pr.name, "sm_clocks_mhz": clocks}


class TimingCache:
    """Measured times (seconds) by device identity and kernel instance."""

    def __init__(self, path, identity):
        self.path = path
        self.device = json.dumps(identity, sort_keys=True)
        self.data = {"devices": {}}
        if path and os.path.exists(path):
            with open(path) as f:
                self.data = json.load(f)
            if not isinstance(self.data.get("devices"), dict):
                raise ValueError("%s is not a timing cache" % path)
        self.entries = self.data["devices"].setdefault(self.device, {})
        self.hits = 0
        self.stored = 0

    @staticmethod
    def key(kernel, params, trials, flush_l2):
        return json.dumps([kernel, sorted((k, float(v)) for k, v in params.items()), int(trials), bool(flush_l2)])

    def get(self, kernel, params, trials, flush_l2):
        v = self.entries.get(self.key(kernel, params, trials, flush_l2))
        if v is not None:
            self.hits += 1
        return v

    def put(self, kernel, params, trials, flush_l2, seconds):
        self.entries[self.key(kernel, params, trials, flush_l2)] = float(seconds)
        self.stored += 1

    def save(self):
        if not self.path:
            return
        tmp = "%s.tmp%d" % (self.path, os.getpid())
        with open(tmp, "w") as f:
            json.dump(self.data, f)
        os.replace(tmp, self.path)
