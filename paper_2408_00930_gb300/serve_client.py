"""Client of a roll-out server in another process (ws_server_listen).

Message marshalling only: a trainer process that holds no GPU context talks to
the serving process over its Unix-domain socket with the messages documented
at ws_server_listen in include/warpsci.h, and receives each chunk's records as
bytes in the ws_fetch layouts.  Every roll-out step runs in the server's CUDA
library.
"""
from __future__ import annotations

import ctypes as C
import socket
import struct

from paper_2408_00930_gb300 import warpsci as W

OP_SUBMIT, OP_WAIT, OP_FETCH, OP_ACK, OP_RELEASE, OP_STATS = 1, 2, 3, 4, 5, 6


class RemoteServer:
    def __init__(self, path: str, timeout_s: float = 300.0):
        self.sock = socket.socket(socket.AF_UNIX, socket.SOCK_STREAM)
        self.sock.settimeout(timeout_s)
        self.sock.connect(path)

    def _send(self, op: int, payload: bytes = b""):
        self.sock.sendall(struct.pack("<II", op, len(payload)) + payload)

    def _recv(self, n: int) -> bytes:
        buf = bytearray()
        while len(buf) < n:
            chunk = self.sock.recv(n - len(buf))
            if not chunk:
                raise ConnectionError("server closed the connection")
            buf += chunk
        return bytes(buf)

    def _status(self) -> int:
        return struct.unpack("<i", self._recv(4))[0]

    def submit(self, q: W.ws_request, agents_per_env=None):
        """Queue a request (a ws_request from warpsci.make_request); returns
        (status, id)."""
        body = bytes(C.string_at(C.addressof(q), C.sizeof(q)))
        if agents_per_env is not None:
            body += struct.pack(f"<{len(agents_per_env)}i", *[int(a) for a in agents_per_env])
        self._send(OP_SUBMIT, body)
        st = self._status()
        (rid,) = struct.unpack("<Q", self._recv(8))
        return st, rid

    def wait_chunk(self, rid: int, chunk: int, timeout_ms: int = 0) -> int:
        self._send(OP_WAIT, struct.pack("<QII", rid, chunk, timeout_ms))
        return self._status()

    def fetch(self, rid: int, field: int, chunk: int):
        """(status, bytes of the field for the chunk's steps)."""
        self._send(OP_FETCH, struct.pack("<QiI", rid, field, chunk))
        st = self._status()
        (n,) = struct.unpack("<Q", self._recv(8))
        return st, self._recv(n) if n else b""

    def ack(self, rid: int, chunk: int) -> int:
        self._send(OP_ACK, struct.pack("<QI", rid, chunk))
        return self._status()

    def release(self, rid: int) -> int:
        self._send(OP_RELEASE, struct.pack("<Q", rid))
        return self._status()

    def stats(self) -> dict:
        self._send(OP_STATS)
        st = self._status()
        if st != W.WS_OK:
            raise W.WarpSciError(st, "stats")
        out = W.ws_server_stats.from_buffer_copy(self._recv(C.sizeof(W.ws_server_stats)))
        return {f: getattr(out, f) for f, _ in W.ws_server_stats._fields_ if f != "struct_size"}

    def close(self):
        try:
            self.sock.close()
        except OSError:
            pass
