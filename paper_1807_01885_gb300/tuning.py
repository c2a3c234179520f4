"""FFT radix choices of the operator passes, tuned once per GPU model, grid size and
precision by the library's autotuner (bem_autotune) and reused by later handles;
optionally kept in a JSON file so that later processes apply them without timing the
passes again.

Orchestration only: the timing itself runs in the library.
"""
import json
import os


def default_path():
    """$BEM_TUNE_CACHE, else ~/.cache/bem_gb300/radix.json."""
    return os.environ.get("BEM_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "bem_gb300",
                                                            "radix.json")


class RadixCache:
    """(log2 row radix, log2 column radix) per (device, N, precision).  ``path``: JSON
    file read at creation and rewritten after every new tuning (None: this process
    only).  ``fixed``: apply these radices to every handle, tuning nothing."""

    def __init__(self, fixed=None, path=None, device=""):
        self.fixed = tuple(fixed) if fixed is not None else None
        self.path = path
        self.device = device
        self.choice = {}
        self.by_size = {}   # grid size -> the radices last applied to a handle of that size
        if path is not None and os.path.exists(path):
            try:
                with open(path) as fh:
                    self.choice = {k: tuple(v) for k, v in json.load(fh).items()}
            except (OSError, ValueError):
                self.choice = {}

    def key(self, k):
        return f"{self.device}|{k.N}|{getattr(k, 'precision', '')}"

    def apply(self, k, stream=None):
        if self.fixed is not None:
            k.set_radix(*self.fixed, stream=stream)
            self.by_size[k.N] = self.fixed
            return self.fixed
        key = self.key(k)
        if key in self.choice:
            k.set_radix(*self.choice[key], stream=stream)
        else:
            self.choice[key] = tuple(k.autotune(reps=5, stream=stream))
            self._write()
        self.by_size[k.N] = self.choice[key]
        return self.choice[key]

    def _write(self):
        if self.path is None:
            return
        os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
        tmp = self.path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump({k: list(v) for k, v in self.choice.items()}, fh, indent=1, sort_keys=True)
        os.replace(tmp, self.path)
