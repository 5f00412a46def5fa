"""A small HDF5 reader for the tests: enough of the file format to walk the
files the map drain writes and to check them value by value.

It is written from the published HDF5 file format (superblock version 0,
version-1 object headers, symbol-table groups with a version-1 B-tree, local
heap and symbol-table nodes; dataspace, datatype, fill value, data layout
version 3, filter pipeline version 1 and attribute messages; chunked storage
indexed by a version-1 B-tree; the deflate, shuffle and LZF filters) and shares
nothing with the writer.  It is checked first on a file written by the HDF5
library itself (a MATLAB 7.3 test file that SciPy ships).
"""
import zlib

import numpy as np

SIGNATURE = b"\x89HDF\r\n\x1a\n"
UNDEF = 0xFFFFFFFFFFFFFFFF


class H5Error(Exception):
    pass


def lzf_decompress(src):
    """LZF stream: a control byte c < 32 is followed by c + 1 literal bytes;
    otherwise length L = c >> 5 (7: plus the next byte) and distance
    ((c & 31) << 8 | next byte) + 1 copy L + 2 bytes from the output."""
    out = bytearray()
    i, n = 0, len(src)
    while i < n:
        c = src[i]
        i += 1
        if c < 32:
            out += src[i:i + c + 1]
            i += c + 1
            continue
        ln = c >> 5
        if ln == 7:
            ln += src[i]
            i += 1
        dist = ((c & 31) << 8 | src[i]) + 1
        i += 1
        if dist > len(out):
            raise H5Error("LZF back reference before the start")
        for _ in range(ln + 2):
            out.append(out[-dist])
    return bytes(out)


class Dataset:
    def __init__(self, name, shape, dtype, attrs, data, filters, chunks):
        self.name, self.shape, self.dtype = name, shape, dtype
        self.attrs, self.data, self.filters, self.chunks = attrs, data, filters, chunks
        self.stored = []  # offsets of the chunks present in the file


class Group:
    def __init__(self, name, attrs):
        self.name, self.attrs, self.members = name, attrs, {}


class File:
    """Parsed file: `root` is a Group; members are Groups or Datasets."""

    def __init__(self, path):
        with open(path, "rb") as f:
            self.d = f.read()
        self.base = self._find_superblock()
        self.root = self._group("/", self._root_header)

    # ----------------------------------------------------------- primitives
    def u(self, off, n):
        return int.from_bytes(self.d[off:off + n], "little")

    def addr(self, a):
        return self.base + a

    def _find_superblock(self):
        # at 0, 512, 1024, 2048, ...
        off = 0
        while off < len(self.d):
            if self.d[off:off + 8] == SIGNATURE:
                break
            off = 512 if off == 0 else off * 2
        else:
            raise H5Error("no HDF5 signature")
        ver = self.d[off + 8]
        if ver != 0:
            raise H5Error("superblock version %d not read here" % ver)
        self.so, self.sl = self.d[off + 13], self.d[off + 14]
        if (self.so, self.sl) != (8, 8):
            raise H5Error("only 8-byte offsets and lengths")
        base = self.u(off + 24, 8)
        ent = off + 56  # root group symbol table entry
        self._root_header = base + self.u(ent + 8, 8)
        return base

    # ------------------------------------------------------ object headers
    def _messages(self, oh):
        """(type, flags, data offset, size) of every message, following
        continuation blocks."""
        if self.d[oh] != 1:
            raise H5Error("object header version %d at %d" % (self.d[oh], oh))
        nmsg = self.u(oh + 2, 2)
        hsize = self.u(oh + 8, 4)
        blocks = [(oh + 16, hsize)]
        out = []
        while blocks and len(out) < nmsg:
            start, size = blocks.pop(0)
            p = start
            while p + 8 <= start + size and len(out) < nmsg:
                mtype, msize, mflags = self.u(p, 2), self.u(p + 2, 2), self.d[p + 4]
                data = p + 8
                if mtype == 0x10:  # continuation
                    blocks.append((self.addr(self.u(data, 8)), self.u(data + 8, 8)))
                out.append((mtype, mflags, data, msize))
                p = data + msize
        return out

    def _dataspace(self, p):
        ver, rank, flags = self.d[p], self.d[p + 1], self.d[p + 2]
        q = p + (8 if ver == 1 else 4)
        if ver == 2 and self.d[p + 3] == 0:  # scalar
            return ()
        return tuple(self.u(q + 8 * i, 8) for i in range(rank))

    def _datatype(self, p):
        cls, ver = self.d[p] & 0x0F, self.d[p] >> 4
        bits = self.d[p + 1] | (self.d[p + 2] << 8) | (self.d[p + 3] << 16)
        size = self.u(p + 4, 4)
        if ver not in (1, 2, 3):
            raise H5Error("datatype version %d" % ver)
        order = ">" if bits & 1 else "<"
        if cls == 0:  # fixed point
            signed = bool(bits & 0x08)
            return np.dtype("%s%s%d" % (order, "i" if signed else "u", size))
        if cls == 1:  # floating point
            return np.dtype("%sf%d" % (order, size))
        if cls == 3:  # string
            return np.dtype("S%d" % size)
        raise H5Error("datatype class %d not read here" % cls)

    def _attribute(self, p):
        ver = self.d[p]
        if ver != 1:
            raise H5Error("attribute message version %d" % ver)
        nsize, tsize, ssize = self.u(p + 2, 2), self.u(p + 4, 2), self.u(p + 6, 2)

        def pad8(n):
            return (n + 7) & ~7

        q = p + 8
        name = self.d[q:q + nsize].split(b"\0")[0].decode()
        q += pad8(nsize)
        dt = self._datatype(q)
        q += pad8(tsize)
        shape = self._dataspace(q)
        q += pad8(ssize)
        n = int(np.prod(shape)) if shape else 1
        val = np.frombuffer(self.d, dt, n, q).reshape(shape) if n else np.zeros(0, dt)
        return name, val

    def _filters(self, p):
        ver, nf = self.d[p], self.d[p + 1]
        if ver != 1:
            raise H5Error("filter pipeline version %d" % ver)
        q = p + 8
        out = []
        for _ in range(nf):
            fid, nlen, flags, ncd = (self.u(q, 2), self.u(q + 2, 2), self.u(q + 4, 2),
                                     self.u(q + 6, 2))
            q += 8 + ((nlen + 7) & ~7)
            cd = [self.u(q + 4 * i, 4) for i in range(ncd)]
            q += 4 * ncd + (4 if ncd % 2 else 0)
            out.append((fid, flags, cd))
        return out

    # ------------------------------------------------------------- storage
    def _unfilter(self, raw, filters, mask, itemsize):
        buf = raw
        for k in reversed(range(len(filters))):
            fid = filters[k][0]
            if mask & (1 << k):
                continue
            if fid == 1:
                buf = zlib.decompress(buf)
            elif fid == 32000:
                buf = lzf_decompress(buf)
            elif fid == 2:  # shuffle: bytes grouped by position within the element
                n = len(buf) // itemsize
                a = np.frombuffer(buf[:n * itemsize], np.uint8).reshape(itemsize, n)
                buf = a.T.tobytes() + buf[n * itemsize:]
            else:
                raise H5Error("filter %d not read here" % fid)
        return buf

    def _chunks(self, tree, rank):
        """Leaf entries (offsets, size, filter mask, address) of a type-1 B-tree."""
        t = self.addr(tree)
        if self.d[t:t + 4] != b"TREE" or self.d[t + 4] != 1:
            raise H5Error("chunk B-tree expected at %d" % t)
        level, used = self.d[t + 5], self.u(t + 6, 2)
        q = t + 24
        ksize = 8 + 8 * (rank + 1)
        out = []
        for i in range(used):
            size, fmask = self.u(q, 4), self.u(q + 4, 4)
            offs = tuple(self.u(q + 8 + 8 * j, 8) for j in range(rank))
            child = self.u(q + ksize, 8)
            q += ksize + 8
            if level == 0:
                out.append((offs, size, fmask, child))
            else:
                out.extend(self._chunks(child, rank))
        return out

    def _dataset(self, name, msgs):
        shape = dtype = layout = None
        filters, attrs, fill = [], {}, None
        for mtype, _, p, _ in msgs:
            if mtype == 0x01:
                shape = self._dataspace(p)
            elif mtype == 0x03:
                dtype = self._datatype(p)
            elif mtype == 0x08:
                layout = p
            elif mtype == 0x05 and self.d[p] == 2 and self.d[p + 3] == 1:
                fill = (p + 8, self.u(p + 4, 4))
            elif mtype == 0x0B:
                filters = self._filters(p)
            elif mtype == 0x0C:
                k, v = self._attribute(p)
                attrs[k] = v
        ver, cls = self.d[layout], self.d[layout + 1]
        n = int(np.prod(shape)) if shape else 1
        chunks = None
        if ver in (1, 2):  # older layout: rank, class, 5 reserved, address, dims
            nd, cls = self.d[layout + 1], self.d[layout + 2]
            if cls != 1:
                raise H5Error("layout version %d class %d not read here" % (ver, cls))
            a = self.u(layout + 8, 8)
            data = np.frombuffer(self.d, dtype, n, self.addr(a)) if a != UNDEF else \
                np.zeros(n, dtype)
            return Dataset(name, shape, dtype, attrs, np.asarray(data).reshape(shape), filters,
                           chunks)
        if ver != 3:
            raise H5Error("data layout version %d not read here" % ver)
        if cls == 0:  # compact
            size = self.u(layout + 2, 2)
            data = np.frombuffer(self.d, dtype, n, layout + 4)
        elif cls == 1:  # contiguous
            a, size = self.u(layout + 2, 8), self.u(layout + 10, 8)
            data = (np.frombuffer(self.d, dtype, n, self.addr(a)) if a != UNDEF
                    else np.zeros(n, dtype))
        elif cls == 2:  # chunked
            nd = self.d[layout + 2]
            tree = self.u(layout + 3, 8)
            cdims = tuple(self.u(layout + 11 + 4 * i, 4) for i in range(nd))
            chunks = cdims[:-1]
            arr = np.zeros(shape, dtype)
            stored = []
            if fill is not None:
                arr[...] = np.frombuffer(self.d, dtype, 1, fill[0])[0]
            if tree != UNDEF:
                for offs, size, fmask, a in self._chunks(tree, len(shape)):
                    stored.append(offs)
                    raw = self.d[self.addr(a):self.addr(a) + size]
                    buf = self._unfilter(raw, filters, fmask, dtype.itemsize)
                    blk = np.frombuffer(buf, dtype, int(np.prod(chunks))).reshape(chunks)
                    sl = tuple(slice(o, min(o + c, s)) for o, c, s in zip(offs, chunks, shape))
                    arr[sl] = blk[tuple(slice(0, s.stop - s.start) for s in sl)]
            data = arr
        else:
            raise H5Error("layout class %d" % cls)
        ds = Dataset(name, shape, dtype, attrs, np.asarray(data).reshape(shape), filters, chunks)
        if cls == 2:
            ds.stored = stored
        return ds

    def _group(self, name, oh):
        msgs = self._messages(oh)
        attrs = {}
        stab = None
        for mtype, _, p, _ in msgs:
            if mtype == 0x11:
                stab = (self.u(p, 8), self.u(p + 8, 8))
            elif mtype == 0x0C:
                k, v = self._attribute(p)
                attrs[k] = v
        if stab is None:
            raise H5Error("object %s is not a symbol-table group" % name)
        g = Group(name, attrs)
        heap = self.addr(stab[1])
        if self.d[heap:heap + 4] != b"HEAP":
            raise H5Error("local heap expected")
        hdata = self.addr(self.u(heap + 24, 8))
        for ent_name, child in self._group_entries(stab[0], hdata):
            cm = self._messages(child)
            types = {m[0] for m in cm}
            full = name.rstrip("/") + "/" + ent_name
            if 0x11 in types:
                g.members[ent_name] = self._group(full, child)
            else:
                g.members[ent_name] = self._dataset(full, cm)
        return g

    def _group_entries(self, tree, hdata):
        t = self.addr(tree)
        if self.d[t:t + 4] != b"TREE" or self.d[t + 4] != 0:
            raise H5Error("group B-tree expected")
        level, used = self.d[t + 5], self.u(t + 6, 2)
        q = t + 24 + 8  # key 0
        out = []
        for i in range(used):
            child = self.addr(self.u(q, 8))
            q += 16  # child, next key
            if level > 0:
                out.extend(self._group_entries(child - self.base, hdata))
                continue
            if self.d[child:child + 4] != b"SNOD":
                raise H5Error("symbol table node expected")
            ns = self.u(child + 6, 2)
            for k in range(ns):
                e = child + 8 + 40 * k
                off = self.u(e, 8)
                nm = self.d[hdata + off:self.d.index(b"\0", hdata + off)].decode()
                out.append((nm, self.addr(self.u(e + 8, 8))))
        return out


def walk(g, prefix=""):
    """(path, Dataset) for every dataset below group g."""
    for k, v in g.members.items():
        path = prefix + "/" + k
        if isinstance(v, Group):
            yield from walk(v, path)
        else:
            yield path, v
