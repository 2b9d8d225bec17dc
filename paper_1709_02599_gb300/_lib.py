"""ctypes declarations of libdls.so (include/dls.h).  Loading fails loudly if
the library has not been built -- there is no fallback implementation."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdls.so")

DLS_MAX_N = 16
DIAGONAL = 1
VSYM = 2

ORDER_MD_AD_ROWS = 0
ORDER_ROW_MAJOR = 1
ORDER_HOURGLASS = 2
ORDER_HEURISTIC = 3
ORDER_HEURISTIC_SQ = 4

KERNEL_PERSISTENT = 0
KERNEL_PLAIN = 1

RUN_PERSISTENT = 0
RUN_PLAIN = 1
RUN_SNAPSHOT = 2
RUN_PLAIN_SNAPSHOT = 3
RUN_NAMES = {RUN_PERSISTENT: "k_persistent", RUN_PLAIN: "k_plain", RUN_SNAPSHOT: "k_snapshot",
             RUN_PLAIN_SNAPSHOT: "k_plain_snap"}
STEP_NAMES = {0: "per-position", 1: "snapshot, field shifts", 2: "snapshot, byte words",
              3: "snapshot, wide words"}

OK = 0
ERR_CAPACITY = 4
ERR_TIMEOUT = 6
ERR_ABORTED = 7
UNFINISHED = 1 << 63

u8p = ctypes.POINTER(ctypes.c_uint8)
u32p = ctypes.POINTER(ctypes.c_uint32)
u64p = ctypes.POINTER(ctypes.c_uint64)
i64p = ctypes.POINTER(ctypes.c_int64)
vp = ctypes.c_void_p


class U128(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_uint64), ("hi", ctypes.c_uint64)]

    def value(self):
        return (int(self.hi) << 64) | int(self.lo)


class LaunchT(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int),
                ("block_threads", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int),
                ("lanes_per_prefix", ctypes.c_int),
                ("split_pos", ctypes.c_int),
                ("donate", ctypes.c_int),
                ("check_every", ctypes.c_int),
                ("words", ctypes.c_int),
                ("stack", ctypes.c_int),
                ("lookahead", ctypes.c_int),
                ("fuse", ctypes.c_int),
                ("budget", ctypes.c_int64),
                ("stack_cap", ctypes.c_int),
                ("abort_flag", ctypes.c_void_p)]


class LaunchInfo(ctypes.Structure):
    _fields_ = [("run", ctypes.c_int),
                ("words", ctypes.c_int),
                ("block_threads", ctypes.c_int),
                ("grid_blocks", ctypes.c_int),
                ("smem_bytes", ctypes.c_int),
                ("stack_entries", ctypes.c_int),
                ("fused", ctypes.c_int),
                ("step", ctypes.c_int)]


class CountStatus(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int),
                ("prefixes_started", ctypes.c_int64)]


class ServerCfg(ctypes.Structure):
    _fields_ = [("max_jobs", ctypes.c_int),
                ("arena_bytes", ctypes.c_size_t),
                ("chunk_bytes", ctypes.c_size_t),
                ("queue_items", ctypes.c_int64),
                ("max_order", ctypes.c_int),
                ("budget", ctypes.c_int),
                ("block_threads", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int),
                ("items_per_job", ctypes.c_int),
                ("min_backlog", ctypes.c_int),
                ("item_nodes", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("pending", ctypes.c_int64),
                ("active", ctypes.c_int64), ("epochs", ctypes.c_int64),
                ("squares", ctypes.c_uint64), ("lanes", ctypes.c_int64),
                ("device_bytes", ctypes.c_size_t), ("free_arena_bytes", ctypes.c_size_t)]


class DlsError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__("%s: %s (status %d)%s" % (
            what, _strerror(code), code,
            (" [%s]" % last_cuda_error()) if code == 5 else ""))


_lib = None


def load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            "libdls.so is not built (%s); run `python -c \"import __graft_entry__ as g; "
            "g.build()\"` or `python -m paper_1709_02599_gb300.build`" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    c_int, c_u32, c_i64 = ctypes.c_int, ctypes.c_uint32, ctypes.c_int64
    c_int64_t = ctypes.c_int64
    sig = {
        "dls_strerror": (ctypes.c_char_p, [c_int]),
        "dls_last_cuda_error": (ctypes.c_char_p, []),
        "dls_version": (c_int, []),
        "dls_fill_order": (c_int, [c_int, c_u32, c_int, c_int, u8p, c_int,
                                   ctypes.POINTER(c_int)]),
        "dls_order_complete": (c_int, [c_int, c_u32, u8p, c_int, c_int, u8p, c_int,
                                       ctypes.POINTER(c_int)]),
        "dls_order_trim": (c_int, [c_int, c_u32, u8p, c_int, c_int, c_int, u8p, c_int,
                                   ctypes.POINTER(c_int)]),
        "dls_extend_prefixes": (c_int, [c_int, c_u32, u8p, c_int, u8p, c_int, c_i64,
                                        c_int, u8p, c_i64, i64p, i64p]),
        "dls_sample_prefix": (c_int, [c_int, c_u32, u8p, c_int, c_int, u32p, c_i64,
                                      u8p, i64p]),
        "dls_estimate_nodes": (c_int, [c_int, c_u32, u8p, c_int, u8p, c_int,
                                       ctypes.c_uint64, c_int,
                                       ctypes.POINTER(ctypes.c_double)]),
        "dls_multiplier": (U128, [c_int, c_u32]),
        "dls_mul_u64": (U128, [ctypes.c_uint64, U128]),
        "dls_add_u128": (U128, [U128, U128]),
        "dls_count": (c_int, [c_int, c_u32, u8p, c_int, vp, c_int, c_i64, vp, vp, vp]),
        "dls_count_plain": (c_int, [c_int, c_u32, u8p, c_int, vp, c_int, c_i64, vp, vp,
                                    vp]),
        "dls_count_ex": (c_int, [c_int, c_u32, u8p, c_int, vp, c_int, c_i64, vp, vp, vp,
                                 ctypes.POINTER(LaunchT), vp]),
        "dls_describe_launch": (c_int, [c_int, c_u32, u8p, c_int, c_int, c_i64,
                                        ctypes.POINTER(LaunchT), ctypes.POINTER(LaunchInfo)]),
        "dls_count_host": (c_int, [c_int, c_u32, u8p, c_int, vp, c_int, c_i64, vp,
                                   ctypes.POINTER(U128), ctypes.POINTER(LaunchT), vp]),
        "dls_count_host_noalloc": (c_int, [c_int, c_u32, u8p, c_int, vp, c_int, c_i64, vp,
                                           ctypes.POINTER(U128), ctypes.POINTER(LaunchT), vp]),
        "dls_hourglass_classes": (c_int, [c_int, c_u32, u8p, c_int, vp, c_int64_t, vp, vp]),
        "dls_count_weighted": (c_int, [c_int, c_u32, u8p, c_int, vp, c_int, c_i64, vp, vp,
                                       c_int, ctypes.POINTER(U128), ctypes.POINTER(LaunchT),
                                       vp]),
        "dls_release": (None, []),
        "dls_stream_status": (c_int, [vp, ctypes.POINTER(CountStatus)]),
        "dls_server_default_cfg": (None, [ctypes.POINTER(ServerCfg)]),
        "dls_server_create": (c_int, [ctypes.POINTER(ServerCfg), ctypes.POINTER(vp)]),
        "dls_server_submit": (c_int, [vp, c_int, c_u32, u8p, c_int, u8p, c_int, i64p]),
        "dls_server_step": (c_int, [vp]),
        "dls_server_poll": (c_int, [vp, i64p, u64p, c_int, ctypes.POINTER(c_int)]),
        "dls_server_get_stats": (c_int, [vp, ctypes.POINTER(ServerStats)]),
        "dls_server_abort": (c_int, [vp]),
        "dls_server_destroy": (None, [vp]),
        "dls_plan_create": (c_int, [ctypes.POINTER(vp), c_int, c_u32, u8p, c_int, vp,
                                    c_int, c_i64, vp, vp, ctypes.POINTER(LaunchT)]),
        "dls_plan_launch": (c_int, [vp, vp]),
        "dls_plan_status": (c_int, [vp, vp, ctypes.POINTER(CountStatus)]),
        "dls_plan_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def declared_symbols():
    """Function names declared in include/dls.h."""
    import re
    hdr = os.path.join(os.path.dirname(HERE), "include", "dls.h")
    text = open(hdr).read()
    # strip comments
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dls_[a-z0-9_]+)\s*\(", text)))


def _strerror(code):
    try:
        return load().dls_strerror(code).decode()
    except Exception:  # pragma: no cover - only while reporting a load failure
        return "status"


def last_cuda_error():
    return load().dls_last_cuda_error().decode()


def check(code, what):
    if code != OK:
        raise DlsError(code, what)
